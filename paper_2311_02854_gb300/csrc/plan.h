// Plan state of libdmrg: MPS, renormalised environments, the current bond's
// intermediates and sigma work lists, and device buffers.
#pragma once

#include <array>
#include <atomic>
#include <exception>
#include <map>
#include <memory>
#include <thread>
#include <string>
#include <vector>

#include "engine.h"
#include "mlp.h"
#include "tc.h"
#include "symbolic.h"

namespace dmrg {

// fn(0 .. n-1) on up to 16 host threads; the first exception is rethrown
template <typename Fn>
void parallel_for(size_t n, const Fn& fn) {
    const size_t nthr = std::min<size_t>(n, std::max(1u, std::min(16u, std::thread::hardware_concurrency())));
    if (nthr <= 1) {
        for (size_t x = 0; x < n; ++x) fn(x);
        return;
    }
    std::atomic<size_t> next{0};
    std::vector<std::exception_ptr> err(nthr);
    std::vector<std::thread> pool;
    for (size_t t = 0; t < nthr; ++t)
        pool.emplace_back([&, t]() {
            try {
                for (size_t x = next++; x < n; x = next++) fn(x);
            } catch (...) {
                err[t] = std::current_exception();
            }
        });
    for (auto& th : pool) th.join();
    for (auto& e : err)
        if (e) std::rethrow_exception(e);
}


// Block-sparse MPS kept on the host (source of truth for save / renormalise).
struct MPSHost {
    int K = 0, N = 0, twoS = 0, center = 1;
    std::vector<std::vector<std::array<int, 3>>> bonds;                        // (N_L, 2Sz_L, dim)
    std::vector<std::map<std::array<int, 3>, std::vector<double>>> sites;      // (il, n, ir) -> d_l x d_r
    bool read(const std::string& path, std::string& err);
    bool write(const std::string& path) const;
};

// Operand view of a dense matrix stored in buffer `buf`: element (i, j) at
// off + i*ld + j, or off + j*ld + i when tr.  `ident` marks the identity.
// Operators of one stored family with the same block structure are nz
// matrices zstride apart: this one is number z (off includes z * zstride).
struct View {
    int8_t buf = -1;
    int64_t off = 0;
    int ld = 0;
    bool tr = false;
    bool ident = false;
    int32_t z = 0, nz = 1;
    int64_t zstride = 0;
    View T() const {
        View v = *this;
        v.tr = !v.tr;
        return v;
    }
};

// out(m x n) += alpha * P(m x k1) Q(k1 x k2) R(k2 x n)
struct Contrib {
    int out;
    View P, Q, R;
    int m, k1, k2, n;
    double alpha;
    int qsec = -1;  // sigma: wavefunction sector read by Q (for the padded bf16 copy)
    int term = -1;  // sigma: index of the Hamiltonian term the product belongs to
};
struct OutBlock {
    int8_t buf;
    int64_t off;
    int m, n, ldc;
};

// Three-factor products lowered onto the segmented GEMM: chunks of
// (phase 1: first product into scratch, phase 2: fused sum into the outputs).
struct ProductList {
    std::vector<OutBlock> outs;
    std::vector<Contrib> cs;
    std::vector<std::pair<WorkList, WorkList>> chunks;
    double flops = 0.0;  // algorithmic
    int64_t scratch_elems = 0;
    int8_t sbuf = -1;  // buffer id of the phase-1 scratch
    bool tc = false;
    int tile_m = 0, tile_n = 0;  // FP64-engine tile shape of lower() (0: the engine's default)
    bool chunk_per_term = false;  // lower_tma: a new scratch chunk (launch pair) at every term
    void clear();
    // FP64 engine: per-segment alpha, 64x64 tiles
    void lower(int8_t scratch_buf, int8_t ident_buf, int ident_ld, int64_t scratch_cap, int64_t kchunk);
    // tensor-core engine: alpha folded into phase-1 products (or a sign bit), 128x128 tiles;
    // phase-1 products are stored as bf16 pieces with rows padded to 8
    void lower_tc(int8_t scratch_buf, int8_t ident_buf, int ident_ld, int64_t scratch_cap, int64_t kchunk,
                  uint8_t out_mode);
    void upload(cudaStream_t st);
    void run(const BufTable& bt, int nvec, cudaStream_t st);
    void run_tc(const TcBufs& tb, int nvec, int nsplit, cudaStream_t st);
    // TMA-staged tensor-core engine: as lower_tc, with every operand read through
    // a tensor map (maps); phase-1 products of equal shape share a 3-D scratch
    // tensor.  vec_bufs: buffers holding one copy per vector (stride vstride[b],
    // nv copies); the maps are encoded later by maps.encode_upload.
    void lower_tma(int8_t scratch_buf, int8_t ident_buf, int ident_ld, int64_t scratch_cap, int64_t kchunk,
                   uint8_t out_mode, const int64_t* vstride, int nv, int tile_n = 128);
    void run_tma(const TcBufs& tb, int nvec, int nsplit, cudaStream_t st);
    std::vector<std::pair<TmaWorkList, TmaWorkList>> tchunks;
    MapTable maps;
    void release();
};

// Intermediates of a bond or of a renormalisation step (FP64 or bf16 pieces).
struct IntermStore {
    double* d = nullptr;
    __nv_bfloat16* h = nullptr;
    __nv_bfloat16* l = nullptr;
    int64_t n = 0;
};

struct Block {
    BlockLayout lay;
    double* d = nullptr;         // FP64 store
    __nv_bfloat16* h = nullptr;  // bf16 pieces (mixed precision)
    __nv_bfloat16* l = nullptr;
    int64_t n = 0;
    // host tier (a block is immutable once built, so one host copy serves every
    // later eviction): which arrays exist, the pinned copy, and the copy events
    bool has_d = false, has_h = false, has_l = false;
    bool dev = true;               // device arrays allocated
    bool host_valid = false;       // pinned copy written (complete once ev_out has)
    bool evicting = false;         // device arrays freed once ev_out completes
    bool fetching = false;         // device arrays valid once ev_in completes
    char* host = nullptr;
    int64_t host_cap = 0;
    cudaEvent_t ev_out = nullptr;  // copy to host done
    cudaEvent_t ev_use = nullptr;  // the compute stream's last use before an eviction
    cudaEvent_t ev_in = nullptr;   // copy back to the device done
};

struct Plan {
    dmrg_options opt{};
    Integrals I;
    MPSHost mps;
    QN tot;
    int K = 0, N = 0, twoS = 0, D = 0, n_so = 0;
    int nsplit = 0;  // 0: FP64 engine; 1: bf16; 2: bf16 x3 (hi + lo); 3: bf16 x6 (hi + lo + lo2)
    bool oz = false;  // FP64-engine products run on the FP64-accurate tensor-core engine
    // tile shape of the FP64-engine work lists (128 x 64 tiles select the tensor-core engine)
    void f64_tiles(WorkList& w) const {
        w.tile_m = oz ? oz_tile_rows() : 0;
        w.tile_n = oz ? oz_tile_cols() : 0;
    }
    void f64_tiles(struct ProductList& pl) const;
    bool mixed() const { return nsplit > 0; }
    // the operator store exists only as bf16 pieces built on the tensor cores
    // (mixed modes without the FP64 master store)
    bool tc_store() const { return nsplit > 0 && !opt.fp64_store; }
    // the operator store has an FP64 copy (FP64 mode, or mixed with fp64_store)
    bool f64_store() const { return nsplit == 0 || opt.fp64_store; }
    // the `lo` array of a piece buffer holds piece 1, then (three pieces) piece 2
    int lo_pieces() const { return nsplit == 3 ? 2 : 1; }
    cudaStream_t stream = nullptr;
    std::string last_error;
    dmrg_stats_t stats{};
    int64_t dev_bytes = 0, budget = 0;

    std::vector<std::unique_ptr<Block>> left, right;  // left[m]: sites 1..m; right[m]: sites m+1..K

    // current bond
    int bond = -1;
    struct Sector {
        int il, y, ir;
        int64_t off;
        int dl, dr;
        int64_t poff;  // offset in the padded (rows of round8(dr)) copy
    };
    std::vector<Sector> layout;
    std::map<std::pair<int, int>, int> sector_of;  // (il, y) -> sector
    std::vector<int> sector_idx;                    // dense: il * 16 + y -> sector or -1
    int64_t dim = 0, dim_pad = 0;
    SigmaPlan sp;
    IntermStore interm;  // the bond's intermediates
    ProductList sigma_pl, hdiag_pl, sigma_tc;
    ProductList sigma_units_pl;  // FP64 sigma on the FP64 arithmetic units (lowered on demand)
    bool sigma_units_ready = false;
    double* d_scratch = nullptr;
    int64_t n_scratch = 0;
    double* d_ident = nullptr;
    int ident_n = 0;
    double* d_wcoef = nullptr;
    int64_t n_wcoef = 0;

    // mixed precision: bf16 pieces (hi, lo) of scratch, wavefunction,
    // identity, coefficient matrices and intermediates
    __nv_bfloat16 *s_hi = nullptr, *s_lo = nullptr;
    int64_t n_spc = 0;
    __nv_bfloat16 *ps_hi = nullptr, *ps_lo = nullptr;
    int64_t n_ppc = 0;
    __nv_bfloat16 *id_hi = nullptr, *id_lo = nullptr;
    int id_n = 0;
    __nv_bfloat16 *w_hi = nullptr, *w_lo = nullptr;
    int64_t n_wpc = 0;
    SplitJob* d_psi_jobs = nullptr;
    int n_psi_jobs = 0;
    int* d_ctr = nullptr;  // [0] tile counter, [1] device error word
    bool sigma_fp64_ready = false;

    // CUDA graphs of the mixed sigma, per number of vectors in a launch, for the
    // current bond; psi / sigma are staged through fixed buffers
    struct SigmaGraph {
        cudaGraphExec_t exec = nullptr;
        int64_t launches = 0;
    };
    std::map<int, SigmaGraph> sigma_graphs;
    cudaStream_t cap_stream = nullptr;
    double* d_sig_io = nullptr;  // [G x dim in | G x dim out]
    int64_t n_sig_io = 0;
    void drop_graphs();

    // device time of each sigma call: an event pair on the launching stream,
    // read back (without a wait) once the pair has completed
    struct SigmaEvents {
        cudaEvent_t a, b;
        double flops;
        int64_t stages;
    };
    std::vector<SigmaEvents> sig_pending;
    // tile-shape autotuner: sector-size histogram key -> (tile width, phase-2 K-chunk)
    std::map<uint64_t, std::pair<int, int64_t>> tune_cache;
    std::vector<cudaEvent_t> ev_pool;
    cudaEvent_t take_event();
    void collect_sigma_times(bool wait);

    // host-buffer entry point
    double* d_io = nullptr;
    int64_t n_io = 0;
    // guess for the next bond left by decimation (guess_nr vectors)
    double* d_guess = nullptr;
    int64_t n_guess = 0;
    int guess_nr = 0;
    // Davidson workspace
    double* d_dav = nullptr;
    int64_t n_dav = 0;
    // learned preconditioner and the harvesting of its training pairs
    Mlp mlp;
    float* d_mlp_feat = nullptr;  // features (5 per element) and outputs of the current bond
    int64_t n_mlp_feat = 0;
    struct Harvest {
        bool on = false;
        int jd_iters = 40;        // MINRES iterations per correction equation
        double jd_tol = 1e-8;     // relative residual of the correction equation
        int64_t per_solve = 1 << 14;
        int64_t pairs = 0;
    } harvest;

    // host tier of the environment blocks (host_tier option): copy stream,
    // pinned buffers released by freed blocks (reused best fit)
    cudaStream_t copy_stream = nullptr;
    std::vector<std::pair<char*, int64_t>> host_pool;
    int64_t host_bytes = 0;

    double* alloc(int64_t n);
    void free(double*& p, int64_t n);
    __nv_bfloat16* alloc_bf16(int64_t n);
    void free_bf16(__nv_bfloat16*& p, int64_t n);
    __nv_bfloat16* alloc_lo(int64_t n) { return alloc_bf16(lo_pieces() * n); }
    void free_lo(__nv_bfloat16*& p, int64_t n) { free_bf16(p, lo_pieces() * n); }
    // piece 2 of a lo array of n elements per piece (null unless three pieces)
    __nv_bfloat16* lo2(__nv_bfloat16* lo, int64_t n) const { return (nsplit == 3 && lo) ? lo + n : nullptr; }
    void check_device_error();
    ~Plan();
};

inline void Plan::f64_tiles(ProductList& pl) const {
    pl.tile_m = oz ? oz_tile_rows() : 0;
    pl.tile_n = oz ? oz_tile_cols() : 0;
}

}  // namespace dmrg

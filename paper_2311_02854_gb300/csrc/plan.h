// Plan state of libdmrg: MPS, renormalised environments, the current bond's
// intermediates and sigma work lists, and device buffers.
#pragma once

#include <array>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "engine.h"
#include "symbolic.h"

namespace dmrg {

// Block-sparse MPS kept on the host (source of truth for save / renormalise).
struct MPSHost {
    int K = 0, N = 0, twoS = 0, center = 1;
    std::vector<std::vector<std::array<int, 3>>> bonds;                        // (N_L, 2Sz_L, dim)
    std::vector<std::map<std::array<int, 3>, std::vector<double>>> sites;      // (il, n, ir) -> d_l x d_r
    bool read(const std::string& path, std::string& err);
    bool write(const std::string& path) const;
    int bond_dim(int b, int i) const { return bonds[b][i][2]; }
};

// Operand view of a dense matrix stored in buffer `buf`: element (i, j) at
// off + i*ld + j, or off + j*ld + i when tr.  `ident` marks the identity.
struct View {
    int8_t buf = -1;
    int64_t off = 0;
    int ld = 0;
    bool tr = false;
    bool ident = false;
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
    void clear();
    void lower(int8_t scratch_buf, int8_t ident_buf, int ident_ld, int64_t scratch_cap, int64_t kchunk);
    void upload(cudaStream_t st);
    void run(const BufTable& bt, int nvec, cudaStream_t st);
    void release();
};

struct Block {
    BlockLayout lay;
    double* d = nullptr;
    int64_t n = 0;
};

struct Plan {
    dmrg_options opt{};
    Integrals I;
    MPSHost mps;
    QN tot;
    int K = 0, N = 0, twoS = 0, D = 0, n_so = 0;
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
    };
    std::vector<Sector> layout;
    std::map<std::pair<int, int>, int> sector_of;  // (il, y) -> sector
    int64_t dim = 0;
    SigmaPlan sp;
    double* d_interm = nullptr;
    int64_t n_interm = 0;
    ProductList sigma_pl, hdiag_pl;
    double* d_scratch = nullptr;
    int64_t n_scratch = 0;
    double* d_ident = nullptr;
    int ident_n = 0;
    double* d_wcoef = nullptr;
    int64_t n_wcoef = 0;

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

    double* alloc(int64_t n);
    void free(double*& p, int64_t n);
    ~Plan();
};

}  // namespace dmrg

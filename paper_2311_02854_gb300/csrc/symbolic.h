// Host-side planning of the sigma product and of the renormalisation:
// operator families of a block, local (one- and two-site) matrices, and the
// expansion of the Hamiltonian into products O^L (x) O^Y (x) O^R whose block
// factors are stored renormalised operators or integral-weighted sums of them
// ("intermediates", Sec. 2.2).
#pragma once

#include <array>
#include <map>
#include <vector>

#include "common.h"

namespace dmrg {

enum Kind : int8_t { KI = 0, KC = 1, KA = 2, KB = 3, KS = 4, KH = 5 };

// A stored operator of a block: a+_p (KC), a+_p a+_q (KA, p<q), a+_p a_q (KB),
// S_p (KS, p outside the block), H (KH).
struct OpKey {
    int8_t kind = KI;
    int16_t p = -1, q = -1;
    bool operator<(const OpKey& o) const {
        if (kind != o.kind) return kind < o.kind;
        if (p != o.p) return p < o.p;
        return q < o.q;
    }
    bool operator==(const OpKey& o) const { return kind == o.kind && p == o.p && q == o.q; }
};

QN key_dq(const OpKey& k);
inline int kind_parity(int8_t kind) { return (kind == KC || kind == KS) ? 1 : 0; }

// Operators of one (kind, dq) on one block share their block structure and are
// stored as a dense [nops x stride] array (op = row, its blocks back to back).
struct Family {
    int8_t kind = KI;
    QN dq;
    std::vector<OpKey> keys;       // row order
    std::vector<int> pair_of_ket;  // ket sector -> pair index, -1 if none
    std::vector<int> ket, bra;     // per pair
    std::vector<int64_t> off;      // per pair, element offset inside an op
    std::vector<int> ld;           // per pair, row pitch (ket dim rounded up to 8)
    int64_t nnz = 0, stride = 0;
    int64_t base = 0;              // element offset of row 0 in the owning buffer
    int nops() const { return (int)keys.size(); }
};
void layout_family(Family& f, const Basis& b);

// Stored operator set of a block of spin orbitals [lo, hi).
struct BlockLayout {
    Basis basis;
    int lo = 0, hi = 0, n_so = 0;
    std::vector<Family> fams;
    std::map<OpKey, std::pair<int, int>> where;  // key -> (family, row)
    int64_t total = 0;                           // elements
    bool contains(int p) const { return p >= lo && p < hi; }
    void build(const Basis& b, int lo_, int hi_, int n_so_);
    std::pair<int, int> find(const OpKey& k) const {
        auto it = where.find(k);
        return it == where.end() ? std::make_pair(-1, -1) : it->second;
    }
};

// Chemist integrals and the antisymmetrised spin-orbital integrals.
struct Integrals {
    int K = 0;
    std::vector<double> h;    // K*K
    std::vector<double> eri;  // K^4, (pq|rs) at ((p*K+q)*K+r)*K+s
    double e_core = 0.0;
    double hso(int p, int q) const {
        if ((p & 1) != (q & 1)) return 0.0;
        return h[(p >> 1) * K + (q >> 1)];
    }
    double v(int p, int q, int r, int s) const {  // <pq|rs>
        if ((p & 1) != (r & 1) || (q & 1) != (s & 1)) return 0.0;
        return eri[(((int64_t)(p >> 1) * K + (r >> 1)) * K + (q >> 1)) * K + (s >> 1)];
    }
    double w(int p, int q, int r, int s) const { return v(p, q, r, s) - v(p, q, s, r); }
};

// Dense matrix on a local space (4 states of one site, 16 of two sites).
struct LocalOp {
    int dim = 4;
    std::vector<double> m;  // row-major dim x dim
    QN dq;
    int parity = 0;
    double at(int i, int j) const { return m[i * dim + j]; }
};

struct LocalOps {
    std::vector<LocalOp> ops;
    std::map<int, int> transposed;
    int add(const LocalOp& op) {
        ops.push_back(op);
        return (int)ops.size() - 1;
    }
    int transpose(int i);
};

LocalOp local_mul(const LocalOp& a, const LocalOp& b);
LocalOp local_T(const LocalOp& a);
LocalOp local_scale_add(const LocalOp& a, double ca, const LocalOp& b, double cb);
void local_finish(LocalOp& a);  // infer dq and parity from the nonzero pattern

// Exact creation operators of one site (4x4) and of two adjacent sites (16x16).
std::array<LocalOp, 2> site_creators();
std::array<LocalOp, 4> pair_creators();

enum Src : int8_t { SRC_I = 0, SRC_STORE = 1, SRC_INTERM = 2 };

// Reference to a block operator used by a term: identity, a stored operator
// (family, row) of block `owner`, or an intermediate (interm family, row).
struct OpRef {
    int8_t src = SRC_I;
    int8_t owner = 0;  // 0 left block, 1 right block
    bool tr = false;   // use the transpose
    int fam = -1, row = 0;
};

// Integral-weighted sums of the operators of one stored family.
struct IntermFamily {
    int owner = 0, src_fam = -1;
    std::vector<std::vector<std::pair<int, double>>> rows;  // sparse coefficients over src rows
    int64_t base = 0;                                        // element offset in the interm buffer
};

struct Interms {
    std::vector<IntermFamily> fams;
    std::map<std::pair<int, int>, int> by_src;
    // Returns an OpRef to sum_i coef[i] * (owner's family src_fam, row i).
    OpRef add(int owner, int src_fam, const std::vector<std::pair<int, double>>& coefs, bool tr);
    void clear() {
        fams.clear();
        by_src.clear();
    }
};

// sigma term: coef * O^L (x) Y (x) O^R, sign (-1)^{par(Y) n(l) + par(R)(n(l)+n(y))}
struct Term3 {
    double c = 1.0;
    OpRef L;
    int y = -1;
    OpRef R;
};

// renormalisation term of a block grown by one site: coef * (big op) x (site op)
struct Term2 {
    double c = 1.0;
    OpRef X;
    int site = -1;
};

struct RenormTarget {
    OpKey key;
    std::vector<Term2> terms;
};

// Sigma terms at bond (k, k+1) (1-based sites): left block L = spin orbitals
// [0, 2k-2), two sites Y = [2k-2, 2k+2), right block R = [2k+2, 2K).
struct SigmaPlan {
    std::vector<Term3> terms;
    LocalOps y;  // 16x16 matrices
    Interms interms;
    bool normal_left = true;
};
void build_sigma_terms(const Integrals& I, const BlockLayout& L, const BlockLayout& R, int k,
                       SigmaPlan& out);

// Terms producing every stored operator of the grown block.  forward: L (+) site
// k0 (0-based spatial orbital) -> new left block; backward: site k0 (+) R.
struct RenormPlan {
    std::vector<RenormTarget> targets;  // in the new block's (family, row) order
    LocalOps site;                      // 4x4 matrices
    Interms interms;
    bool forward = true;
};
void build_renorm_terms(const Integrals& I, const BlockLayout& big, const BlockLayout& out_layout,
                        int k0, bool forward, RenormPlan& out);

}  // namespace dmrg

// Operator families, local matrices and the symbolic expansion of the
// two-site Hamiltonian (Eq. Sigma) and of the renormalisation (Eq. Renorm).
//
// Derivation used throughout (Sec. 2.3, operators of Eq. qops): for two
// blocks X, Y with every orbital of X before Y in Jordan-Wigner order,
//   H = H^X + H^Y + sum_{p in X}(a+p S^Y_p + h.c.) + sum_{p in Y}(a+p S^X_p + h.c.)
//       + sum_{p<q in N}(A_pq P^M_pq + h.c.) + sum_{p,s in N} B_ps Q^M_ps
// with N the block holding normal operators and M the other, and
//   S^{XY}_p = S^X_p + S^Y_p + sum_{q in X} a+q P^Y_pq + sum_{q in Y} P^X_pq a+q
//            + sum_{r in Y} Q^X_pr a_r + sum_{s in X} a_s Q^Y_ps,
// P_pq = sum_{s<r} <pq||sr> a_r a_s = sum w_pqsr (A_sr)^T, Q_ps = sum w_pqsr B_qr.
// Products are written with operators of the left block first; an operator
// product O^X O^Y then acts on |x y> with the factor (-1)^{par(O^Y) n(x)}
// (the zeta of Eq. Sigma / Eq. Renorm).
#include "symbolic.h"

#include <algorithm>
#include <cmath>
#include <functional>

namespace dmrg {

QN key_dq(const OpKey& k) {
    switch (k.kind) {
        case KC: return {1, spin_of(k.p)};
        case KA: return {2, spin_of(k.p) + spin_of(k.q)};
        case KB: return {0, spin_of(k.p) - spin_of(k.q)};
        case KS: return {-1, -spin_of(k.p)};
        default: return {0, 0};
    }
}

void layout_family(Family& f, const Basis& b) {
    f.pair_of_ket.assign(b.size(), -1);
    f.ket.clear();
    f.bra.clear();
    f.off.clear();
    f.ld.clear();
    int64_t off = 0;
    for (int i = 0; i < b.size(); ++i) {
        int j = b.find(b.qn[i] + f.dq);
        if (j < 0) continue;
        f.pair_of_ket[i] = (int)f.ket.size();
        f.ket.push_back(i);
        f.bra.push_back(j);
        f.off.push_back(off);
        const int ldi = (int)round_up(b.dim[i], 8);  // rows padded to 16 bytes of bf16
        f.ld.push_back(ldi);
        off += (int64_t)b.dim[j] * ldi;
    }
    f.nnz = off;
    f.stride = round_up(std::max<int64_t>(off, 1), 32);
}

void BlockLayout::build(const Basis& b, int lo_, int hi_, int n_so_) {
    basis = b;
    lo = lo_;
    hi = hi_;
    n_so = n_so_;
    fams.clear();
    where.clear();
    std::vector<OpKey> keys;
    for (int p = lo; p < hi; ++p) keys.push_back({KC, (int16_t)p, -1});
    for (int p = lo; p < hi; ++p)
        for (int q = p + 1; q < hi; ++q) keys.push_back({KA, (int16_t)p, (int16_t)q});
    for (int p = lo; p < hi; ++p)
        for (int s = lo; s < hi; ++s) keys.push_back({KB, (int16_t)p, (int16_t)s});
    for (int p = 0; p < n_so; ++p)
        if (!contains(p)) keys.push_back({KS, (int16_t)p, -1});
    keys.push_back({KH, -1, -1});
    std::map<std::pair<int, QN>, int> fidx;
    for (const OpKey& k : keys) {
        QN dq = key_dq(k);
        auto fk = std::make_pair((int)k.kind, dq);
        auto it = fidx.find(fk);
        int f;
        if (it == fidx.end()) {
            f = (int)fams.size();
            fidx[fk] = f;
            fams.emplace_back();
            fams.back().kind = k.kind;
            fams.back().dq = dq;
        } else {
            f = it->second;
        }
        where[k] = {f, fams[f].nops()};
        fams[f].keys.push_back(k);
    }
    total = 0;
    for (Family& f : fams) {
        layout_family(f, basis);
        f.base = total;
        total += f.stride * f.nops();
    }
}

// ---------------------------------------------------------------------------
// Local matrices
// ---------------------------------------------------------------------------

static QN local_qn(int dim, int i) {
    if (dim == 4) return kSiteQN[i];
    return kSiteQN[i / 4] + kSiteQN[i % 4];
}

void local_finish(LocalOp& a) {
    bool have = false;
    QN dq;
    for (int i = 0; i < a.dim; ++i)
        for (int j = 0; j < a.dim; ++j) {
            double x = a.m[i * a.dim + j];
            if (x == 0.0) continue;
            QN d = local_qn(a.dim, i) - local_qn(a.dim, j);
            if (!have) {
                dq = d;
                have = true;
            } else if (d != dq) {
                throw Error(DMRG_EINVAL, "local operator without a definite quantum-number change");
            }
        }
    a.dq = have ? dq : QN{0, 0};
    a.parity = a.dq.n & 1;
}

LocalOp local_mul(const LocalOp& a, const LocalOp& b) {
    LocalOp c;
    c.dim = a.dim;
    c.m.assign(a.dim * a.dim, 0.0);
    for (int i = 0; i < a.dim; ++i)
        for (int k = 0; k < a.dim; ++k) {
            double x = a.m[i * a.dim + k];
            if (x == 0.0) continue;
            for (int j = 0; j < a.dim; ++j) c.m[i * a.dim + j] += x * b.m[k * a.dim + j];
        }
    local_finish(c);
    return c;
}

LocalOp local_T(const LocalOp& a) {
    LocalOp c;
    c.dim = a.dim;
    c.m.assign(a.dim * a.dim, 0.0);
    for (int i = 0; i < a.dim; ++i)
        for (int j = 0; j < a.dim; ++j) c.m[j * a.dim + i] = a.m[i * a.dim + j];
    local_finish(c);
    return c;
}

LocalOp local_scale_add(const LocalOp& a, double ca, const LocalOp& b, double cb) {
    LocalOp c;
    c.dim = a.dim;
    c.m.assign(a.dim * a.dim, 0.0);
    for (int i = 0; i < a.dim * a.dim; ++i) c.m[i] = ca * a.m[i] + cb * b.m[i];
    local_finish(c);
    return c;
}

static LocalOp local_zero(int dim) {
    LocalOp c;
    c.dim = dim;
    c.m.assign(dim * dim, 0.0);
    local_finish(c);
    return c;
}

static LocalOp local_identity(int dim) {
    LocalOp c = local_zero(dim);
    for (int i = 0; i < dim; ++i) c.m[i * dim + i] = 1.0;
    local_finish(c);
    return c;
}

int LocalOps::transpose(int i) {
    auto it = transposed.find(i);
    if (it != transposed.end()) return it->second;
    int j = add(local_T(ops[i]));
    transposed[i] = j;
    transposed[j] = i;
    return j;
}

std::array<LocalOp, 2> site_creators() {
    std::array<LocalOp, 2> c;
    for (auto& x : c) x = local_zero(4);
    c[0].m[2 * 4 + 0] = 1.0;   // a+_a |vac> = |a>
    c[0].m[3 * 4 + 1] = 1.0;   // a+_a |b>   = |ab>
    c[1].m[1 * 4 + 0] = 1.0;   // a+_b |vac> = |b>
    c[1].m[3 * 4 + 2] = -1.0;  // a+_b |a>   = -|ab>
    for (auto& x : c) local_finish(x);
    return c;
}

std::array<LocalOp, 4> pair_creators() {
    auto s = site_creators();
    const double par[4] = {1, -1, -1, 1};
    std::array<LocalOp, 4> c;
    for (auto& x : c) x = local_zero(16);
    for (int sp = 0; sp < 2; ++sp)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                // first site: cd (x) I
                double x = s[sp].m[a * 4 + b];
                if (x != 0.0)
                    for (int t = 0; t < 4; ++t) c[sp].m[(a * 4 + t) * 16 + (b * 4 + t)] = x;
                // second site: parity (x) cd
                if (x != 0.0)
                    for (int t = 0; t < 4; ++t) c[2 + sp].m[(t * 4 + a) * 16 + (t * 4 + b)] = par[t] * x;
            }
    for (auto& x : c) local_finish(x);
    return c;
}

// ---------------------------------------------------------------------------
// Intermediates
// ---------------------------------------------------------------------------

OpRef Interms::add(int owner, int src_fam, const std::vector<std::pair<int, double>>& coefs, bool tr) {
    auto key = std::make_pair(owner, src_fam);
    auto it = by_src.find(key);
    int f;
    if (it == by_src.end()) {
        f = (int)fams.size();
        by_src[key] = f;
        fams.emplace_back();
        fams.back().owner = owner;
        fams.back().src_fam = src_fam;
    } else {
        f = it->second;
    }
    fams[f].rows.push_back(coefs);
    OpRef r;
    r.src = SRC_INTERM;
    r.owner = (int8_t)owner;
    r.tr = tr;
    r.fam = f;
    r.row = (int)fams[f].rows.size() - 1;
    return r;
}

// ---------------------------------------------------------------------------
// Expansion helpers
// ---------------------------------------------------------------------------

namespace {

// A list of operators of one kind on one block (identity: one entry).
struct OpList {
    int owner = 0;
    int8_t kind = KI;
    bool tr = false;
    std::vector<OpKey> keys;
};

OpList ident(int owner) {
    OpList l;
    l.owner = owner;
    l.kind = KI;
    l.keys.push_back(OpKey{});
    return l;
}

OpList list_C(const BlockLayout& B, int owner, bool tr) {
    OpList l;
    l.owner = owner;
    l.kind = KC;
    l.tr = tr;
    for (int p = B.lo; p < B.hi; ++p) l.keys.push_back({KC, (int16_t)p, -1});
    return l;
}

OpList list_A(const BlockLayout& B, int owner, bool tr) {
    OpList l;
    l.owner = owner;
    l.kind = KA;
    l.tr = tr;
    for (int p = B.lo; p < B.hi; ++p)
        for (int q = p + 1; q < B.hi; ++q) l.keys.push_back({KA, (int16_t)p, (int16_t)q});
    return l;
}

OpList list_B(const BlockLayout& B, int owner, bool tr) {
    OpList l;
    l.owner = owner;
    l.kind = KB;
    l.tr = tr;
    for (int p = B.lo; p < B.hi; ++p)
        for (int s = B.lo; s < B.hi; ++s) l.keys.push_back({KB, (int16_t)p, (int16_t)s});
    return l;
}

OpRef ref_store(const BlockLayout& B, int owner, const OpKey& k, bool tr) {
    OpRef r;
    if (k.kind == KI) return r;
    auto fr = B.find(k);
    if (fr.first < 0) throw Error(DMRG_EINVAL, "operator missing from block store");
    r.src = SRC_STORE;
    r.owner = (int8_t)owner;
    r.tr = tr;
    r.fam = fr.first;
    r.row = fr.second;
    return r;
}

QN list_dq(const OpList& l, int i) {
    if (l.kind == KI) return {0, 0};
    QN d = key_dq(l.keys[i]);
    return l.tr ? -d : d;
}

OpRef flip(OpRef r) {
    if (r.src != SRC_I) r.tr = !r.tr;
    return r;
}

struct Expander {
    const Integrals& I;
    const BlockLayout* blocks[2];
    Interms& interms;
    LocalOps& loc;

    OpRef contract(const OpList& l, const std::vector<std::pair<int, double>>& coefs) {
        // sum_i coefs * l[i]; all entries of one list with one dq share a family
        const BlockLayout& B = *blocks[l.owner];
        int fam = -1;
        std::vector<std::pair<int, double>> rows;
        for (auto& ic : coefs) {
            auto fr = B.find(l.keys[ic.first]);
            if (fam < 0) fam = fr.first;
            if (fr.first != fam) throw Error(DMRG_EINVAL, "intermediate spans families");
            rows.push_back({fr.second, ic.second});
        }
        return interms.add(l.owner, fam, rows, l.tr);
    }
};

int parity_of(const OpList& l) { return kind_parity(l.kind); }

}  // namespace

// ---------------------------------------------------------------------------
// Sigma terms
// ---------------------------------------------------------------------------

namespace {

struct SigmaBuilder : Expander {
    SigmaPlan& P;
    SigmaBuilder(const Integrals& I_, const BlockLayout& L, const BlockLayout& R, SigmaPlan& P_)
        : Expander{I_, {&L, &R}, P_.interms, P_.y}, P(P_) {}

    void push(double c, OpRef L, int y, OpRef R, bool hc, int pL, int pR) {
        if (c == 0.0) return;
        P.terms.push_back({c, L, y, R});
        if (hc) {
            int pY = loc.ops[y].parity;
            int e = pL * pY + pL * pR + pY * pR;
            double sgn = (e & 1) ? -1.0 : 1.0;
            P.terms.push_back({c * sgn, flip(L), loc.transpose(y), flip(R)});
        }
    }

    // sum_{i,j} W(i,j) L[i] (x) Y (x) R[j], grouped into terms with
    // intermediates on whichever side gives fewer terms.
    void klass(double c0, const OpList& L, int y, const OpList& R,
               const std::function<double(int, int)>& W, bool hc) {
        QN dqY = loc.ops[y].dq;
        bool zeroY = true;
        for (double x : loc.ops[y].m) zeroY = zeroY && (x == 0.0);
        if (zeroY) return;
        std::map<QN, std::vector<int>> gl, gr;
        for (int i = 0; i < (int)L.keys.size(); ++i) gl[list_dq(L, i)].push_back(i);
        for (int j = 0; j < (int)R.keys.size(); ++j) gr[list_dq(R, j)].push_back(j);
        int pL = parity_of(L), pR = parity_of(R);
        for (auto& a : gl)
            for (auto& b : gr) {
                bool conserving = (a.first + dqY + b.first) == QN(0, 0);
                std::vector<int> rows_nz, cols_nz;
                std::vector<char> colmark(b.second.size(), 0);
                for (int i : a.second) {
                    bool any = false;
                    for (size_t jj = 0; jj < b.second.size(); ++jj) {
                        if (W(i, b.second[jj]) != 0.0) {
                            any = true;
                            colmark[jj] = 1;
                        }
                    }
                    if (any) rows_nz.push_back(i);
                }
                if (rows_nz.empty()) continue;
                if (!conserving) throw Error(DMRG_EINVAL, "symmetry-breaking term in the Hamiltonian");
                for (size_t jj = 0; jj < b.second.size(); ++jj)
                    if (colmark[jj]) cols_nz.push_back(b.second[jj]);
                if (rows_nz.size() <= cols_nz.size()) {
                    for (int i : rows_nz) {
                        std::vector<std::pair<int, double>> cf;
                        for (int j : cols_nz) {
                            double x = W(i, j);
                            if (x != 0.0) cf.push_back({j, x});
                        }
                        OpRef lr = ref_store(*blocks[L.owner], L.owner, L.keys[i], L.tr);
                        if (cf.size() == 1) {
                            OpRef rr = ref_store(*blocks[R.owner], R.owner, R.keys[cf[0].first], R.tr);
                            push(c0 * cf[0].second, lr, y, rr, hc, pL, pR);
                        } else {
                            push(c0, lr, y, contract(R, cf), hc, pL, pR);
                        }
                    }
                } else {
                    for (int j : cols_nz) {
                        std::vector<std::pair<int, double>> cf;
                        for (int i : rows_nz) {
                            double x = W(i, j);
                            if (x != 0.0) cf.push_back({i, x});
                        }
                        OpRef rr = ref_store(*blocks[R.owner], R.owner, R.keys[j], R.tr);
                        if (cf.size() == 1) {
                            OpRef lr = ref_store(*blocks[L.owner], L.owner, L.keys[cf[0].first], L.tr);
                            push(c0 * cf[0].second, lr, y, rr, hc, pL, pR);
                        } else {
                            push(c0, contract(L, cf), y, rr, hc, pL, pR);
                        }
                    }
                }
            }
    }
};

}  // namespace

void build_sigma_terms(const Integrals& I, const BlockLayout& L, const BlockLayout& R, int k,
                       SigmaPlan& P) {
    P.terms.clear();
    P.interms.clear();
    P.y = LocalOps();
    SigmaBuilder sb(I, L, R, P);
    auto cyc = pair_creators();
    const int y0 = 2 * (k - 1);
    int yo[4] = {y0, y0 + 1, y0 + 2, y0 + 3};
    LocalOp cy[4], an[4];
    for (int i = 0; i < 4; ++i) {
        cy[i] = cyc[i];
        an[i] = local_T(cyc[i]);
    }
    auto Y = [&](const LocalOp& m) { return P.y.add(m); };
    const int yI = Y(local_identity(16));
    const OpList IL = ident(0), IR = ident(1);
    const int nL = L.hi - L.lo, nR = R.hi - R.lo;
    P.normal_left = (nL <= nR);

    auto kC = [](int p) { return OpKey{KC, (int16_t)p, -1}; };
    auto kS = [](int p) { return OpKey{KS, (int16_t)p, -1}; };
    const OpKey kH{KH, -1, -1};

    // two-site Hamiltonian H^Y (exact, 16x16)
    {
        LocalOp H = local_zero(16);
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                double x = I.hso(yo[a], yo[b]);
                if (x != 0.0) H = local_scale_add(H, 1.0, local_mul(cy[a], an[b]), x);
            }
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b)
                for (int c = 0; c < 4; ++c)
                    for (int d = c + 1; d < 4; ++d) {
                        double x = I.w(yo[a], yo[b], yo[c], yo[d]);
                        if (x == 0.0) continue;
                        LocalOp t = local_mul(local_mul(cy[a], cy[b]), local_mul(an[d], an[c]));
                        H = local_scale_add(H, 1.0, t, x);
                    }
        sb.push(1.0, OpRef{}, Y(H), OpRef{}, false, 0, 0);
    }
    // H^L, H^R
    sb.push(1.0, ref_store(L, 0, kH, false), yI, OpRef{}, false, 0, 0);
    sb.push(1.0, OpRef{}, yI, ref_store(R, 1, kH, false), false, 0, 0);

    // elementary decomposition of S^Y_p: (matrix, coef(p))
    std::vector<std::pair<int, std::function<double(int)>>> SYel;
    for (int a = 0; a < 4; ++a) {
        int q = yo[a];
        SYel.push_back({Y(an[a]), [&I, q](int p) { return 0.5 * I.hso(p, q); }});
    }
    for (int a = 0; a < 4; ++a)
        for (int s = 0; s < 4; ++s)
            for (int r = s + 1; r < 4; ++r) {
                int q = yo[a], os = yo[s], orr = yo[r];
                LocalOp m = local_mul(cy[a], local_mul(an[r], an[s]));
                SYel.push_back({Y(m), [&I, q, os, orr](int p) { return I.w(p, q, os, orr); }});
            }

    // --- Lambda | R : one index in Lambda, three in R:  a+_p S^R_p + h.c.
    for (int p = L.lo; p < L.hi; ++p)
        sb.push(1.0, ref_store(L, 0, kC(p), false), yI, ref_store(R, 1, kS(p), false), true, 1, 1);
    for (int a = 0; a < 4; ++a) sb.push(1.0, OpRef{}, Y(cy[a]), ref_store(R, 1, kS(yo[a]), false), true, 0, 1);

    // --- three indices in Lambda, one in R: -S^Lambda_p a+^R_p + h.c.
    const OpList CR = list_C(R, 1, false);
    const OpList CL = list_C(L, 0, false), CLt = list_C(L, 0, true);
    const OpList AL = list_A(L, 0, false), ALt = list_A(L, 0, true);
    const OpList BL = list_B(L, 0, false);
    const OpList AR = list_A(R, 1, false), ARt = list_A(R, 1, true);
    const OpList BR = list_B(R, 1, false);
    auto Rp = [&](int j) { return (int)CR.keys[j].p; };
    auto Lp = [&](const OpList& l, int i) { return (int)l.keys[i].p; };
    auto Lq = [&](const OpList& l, int i) { return (int)l.keys[i].q; };
    for (int p = R.lo; p < R.hi; ++p)
        sb.push(-1.0, ref_store(L, 0, kS(p), false), yI, ref_store(R, 1, kC(p), false), true, 1, 1);
    for (auto& e : SYel) {
        auto f = e.second;
        sb.klass(-1.0, IL, e.first, CR, [&](int, int j) { return f(Rp(j)); }, true);
    }
    for (int s = 0; s < 4; ++s)
        for (int r = s + 1; r < 4; ++r) {
            int y = Y(local_mul(an[r], an[s]));
            int os = yo[s], orr = yo[r];
            sb.klass(-1.0, CL, y, CR, [&](int i, int j) { return I.w(Rp(j), Lp(CL, i), os, orr); }, true);
        }
    for (int a = 0; a < 4; ++a) {
        int q = yo[a];
        sb.klass(-1.0, ALt, Y(cy[a]), CR,
                 [&](int i, int j) { return I.w(Rp(j), q, Lp(ALt, i), Lq(ALt, i)); }, true);
    }
    for (int a = 0; a < 4; ++a) {
        int r = yo[a];
        sb.klass(-1.0, BL, Y(an[a]), CR,
                 [&](int i, int j) { return I.w(Rp(j), Lp(BL, i), r, Lq(BL, i)); }, true);
    }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            int q = yo[a], r = yo[b];
            int y = Y(local_mul(cy[a], an[b]));
            sb.klass(-1.0, CLt, y, CR, [&](int i, int j) { return I.w(Rp(j), q, Lp(CLt, i), r); }, true);
        }

    // --- two indices in Lambda, two in R
    if (P.normal_left) {
        sb.klass(1.0, AL, yI, ARt,
                 [&](int i, int j) { return I.w(Lp(AL, i), Lq(AL, i), Lp(ARt, j), Lq(ARt, j)); }, true);
        for (int a = 0; a < 4; ++a) {
            int q = yo[a];
            sb.klass(1.0, CL, Y(cy[a]), ARt,
                     [&](int i, int j) { return I.w(Lp(CL, i), q, Lp(ARt, j), Lq(ARt, j)); }, true);
        }
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b) {
                int p = yo[a], q = yo[b];
                int y = Y(local_mul(cy[a], cy[b]));
                sb.klass(1.0, IL, y, ARt, [&](int, int j) { return I.w(p, q, Lp(ARt, j), Lq(ARt, j)); }, true);
            }
        sb.klass(1.0, BL, yI, BR,
                 [&](int i, int j) { return I.w(Lp(BL, i), Lp(BR, j), Lq(BL, i), Lq(BR, j)); }, false);
        for (int a = 0; a < 4; ++a) {
            int s = yo[a];
            sb.klass(1.0, CL, Y(an[a]), BR,
                     [&](int i, int j) { return I.w(Lp(CL, i), Lp(BR, j), s, Lq(BR, j)); }, false);
        }
        for (int a = 0; a < 4; ++a) {
            int p = yo[a];
            sb.klass(1.0, CLt, Y(cy[a]), BR,
                     [&](int i, int j) { return -I.w(p, Lp(BR, j), Lp(CLt, i), Lq(BR, j)); }, false);
        }
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                int p = yo[a], s = yo[b];
                int y = Y(local_mul(cy[a], an[b]));
                sb.klass(1.0, IL, y, BR, [&](int, int j) { return I.w(p, Lp(BR, j), s, Lq(BR, j)); }, false);
            }
    } else {
        sb.klass(1.0, ALt, yI, AR,
                 [&](int i, int j) { return I.w(Lp(AR, j), Lq(AR, j), Lp(ALt, i), Lq(ALt, i)); }, true);
        for (int s = 0; s < 4; ++s)
            for (int r = s + 1; r < 4; ++r) {
                int os = yo[s], orr = yo[r];
                int y = Y(local_mul(an[r], an[s]));
                sb.klass(1.0, IL, y, AR, [&](int, int j) { return I.w(Lp(AR, j), Lq(AR, j), os, orr); }, true);
            }
        for (int a = 0; a < 4; ++a) {
            int r = yo[a];
            sb.klass(1.0, CLt, Y(an[a]), AR,
                     [&](int i, int j) { return -I.w(Lp(AR, j), Lq(AR, j), Lp(CLt, i), r); }, true);
        }
        sb.klass(1.0, BL, yI, BR,
                 [&](int i, int j) { return I.w(Lp(BR, j), Lp(BL, i), Lq(BR, j), Lq(BL, i)); }, false);
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                int q = yo[a], r = yo[b];
                int y = Y(local_mul(cy[a], an[b]));
                sb.klass(1.0, IL, y, BR, [&](int, int j) { return I.w(Lp(BR, j), q, Lq(BR, j), r); }, false);
            }
        for (int a = 0; a < 4; ++a) {
            int r = yo[a];
            sb.klass(1.0, CL, Y(an[a]), BR,
                     [&](int i, int j) { return I.w(Lp(BR, j), Lp(CL, i), Lq(BR, j), r); }, false);
        }
        for (int a = 0; a < 4; ++a) {
            int q = yo[a];
            sb.klass(1.0, CLt, Y(cy[a]), BR,
                     [&](int i, int j) { return -I.w(Lp(BR, j), q, Lq(BR, j), Lp(CLt, i)); }, false);
        }
    }

    // --- L | Y interactions inside Lambda (normal operators on the two sites)
    for (auto& e : SYel) {
        auto f = e.second;
        sb.klass(1.0, CL, e.first, IR, [&](int i, int) { return f(Lp(CL, i)); }, true);
    }
    for (int a = 0; a < 4; ++a)
        sb.push(-1.0, ref_store(L, 0, kS(yo[a]), false), Y(cy[a]), OpRef{}, true, 1, 0);
    for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b) {
            int p = yo[a], q = yo[b];
            int y = Y(local_mul(cy[a], cy[b]));
            sb.klass(1.0, ALt, y, IR, [&](int i, int) { return I.w(p, q, Lp(ALt, i), Lq(ALt, i)); }, true);
        }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            int p = yo[a], s = yo[b];
            int y = Y(local_mul(cy[a], an[b]));
            sb.klass(1.0, BL, y, IR, [&](int i, int) { return I.w(p, Lp(BL, i), s, Lq(BL, i)); }, false);
        }
}

// ---------------------------------------------------------------------------
// Renormalisation terms
// ---------------------------------------------------------------------------

namespace {

struct RenormBuilder : Expander {
    RenormPlan& P;
    const BlockLayout& big;
    RenormBuilder(const Integrals& I_, const BlockLayout& B, RenormPlan& P_)
        : Expander{I_, {&B, &B}, P_.interms, P_.site}, P(P_), big(B) {}

    OpRef st(const OpKey& k, bool tr = false) { return ref_store(big, 0, k, tr); }
    OpRef lin(const OpList& l, const std::function<double(int)>& coef) {
        std::vector<std::pair<int, double>> cf;
        for (int i = 0; i < (int)l.keys.size(); ++i) {
            double x = coef(i);
            if (x != 0.0) cf.push_back({i, x});
        }
        if (cf.empty()) return OpRef{SRC_I, 0, false, -2, 0};  // marker: zero
        if (cf.size() == 1 && cf[0].second == 1.0) return ref_store(big, 0, l.keys[cf[0].first], l.tr);
        return contract(l, cf);
    }
};

bool is_zero_ref(const OpRef& r) { return r.src == SRC_I && r.fam == -2; }

}  // namespace

void build_renorm_terms(const Integrals& I, const BlockLayout& big, const BlockLayout& out,
                        int k0, bool fwd, RenormPlan& P) {
    P.targets.clear();
    P.interms.clear();
    P.site = LocalOps();
    P.forward = fwd;
    RenormBuilder rb(I, big, P);
    auto sc = site_creators();
    const int c0 = 2 * k0;
    int co[2] = {c0, c0 + 1};
    LocalOp cd[2] = {sc[0], sc[1]}, an[2] = {local_T(sc[0]), local_T(sc[1])};
    auto S = [&](const LocalOp& m) { return P.site.add(m); };
    const int sI = S(local_identity(4));
    int s_cd[2] = {S(cd[0]), S(cd[1])}, s_an[2] = {S(an[0]), S(an[1])};
    auto site_of = [&](int p) { return p - c0; };  // 0 or 1
    auto inC = [&](int p) { return p == c0 || p == c0 + 1; };
    const OpList CB = list_C(big, 0, false), CBt = list_C(big, 0, true);
    const OpList AB = list_A(big, 0, false), ABt = list_A(big, 0, true);
    const OpList BB = list_B(big, 0, false);
    auto P_ = [&](const OpList& l, int i) { return (int)l.keys[i].p; };
    auto Q_ = [&](const OpList& l, int i) { return (int)l.keys[i].q; };

    // exact site operators
    LocalOp HC = local_zero(4);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            double x = I.hso(co[a], co[b]);
            if (x != 0.0) HC = local_scale_add(HC, 1.0, local_mul(cd[a], an[b]), x);
        }
    {
        double x = I.w(co[0], co[1], co[0], co[1]);
        if (x != 0.0) HC = local_scale_add(HC, 1.0, local_mul(local_mul(cd[0], cd[1]), local_mul(an[1], an[0])), x);
    }
    const LocalOp AC = local_mul(cd[0], cd[1]);       // a+_a a+_b
    const LocalOp aa = local_mul(an[1], an[0]);       // a_b a_a
    auto SC_full = [&](int p) {  // S^C_p = sum_q 1/2 h_pq a_q + sum_q w_{pq,ab} a+_q a_b a_a
        LocalOp m = local_zero(4);
        for (int a = 0; a < 2; ++a) {
            double x = 0.5 * I.hso(p, co[a]);
            if (x != 0.0) m = local_scale_add(m, 1.0, an[a], x);
            double y = I.w(p, co[a], co[0], co[1]);
            if (y != 0.0) m = local_scale_add(m, 1.0, local_mul(cd[a], aa), y);
        }
        return m;
    };
    // elementary pieces of S^C_p: (site matrix, coefficient as a function of p)
    std::vector<std::pair<int, std::function<double(int)>>> SCel;
    for (int a = 0; a < 2; ++a) {
        int q = co[a];
        SCel.push_back({S(an[a]), [&I, q](int p) { return 0.5 * I.hso(p, q); }});
        SCel.push_back({S(local_mul(cd[a], aa)), [&I, q, c0](int p) { return I.w(p, q, c0, c0 + 1); }});
    }

    auto add = [&](RenormTarget& t, double c, OpRef X, int site) {
        if (c == 0.0 || is_zero_ref(X)) return;
        if (!(X.src == SRC_I) || true) t.terms.push_back({c, X, site});
    };
    auto addS = [&](RenormTarget& t, double c, OpRef X, const LocalOp& m) {
        bool z = true;
        for (double v : m.m) z = z && v == 0.0;
        if (!z) add(t, c, X, S(m));
    };
    const OpRef Iref{};

    for (const Family& f : out.fams) {
        for (const OpKey& key : f.keys) {
            RenormTarget t;
            t.key = key;
            int p = key.p, q = key.q;
            switch (key.kind) {
                case KC:
                    if (inC(p)) add(t, 1.0, Iref, s_cd[site_of(p)]);
                    else add(t, 1.0, rb.st(key), sI);
                    break;
                case KA:
                    if (inC(p) && inC(q)) addS(t, 1.0, Iref, local_mul(cd[site_of(p)], cd[site_of(q)]));
                    else if (!inC(p) && !inC(q)) add(t, 1.0, rb.st(key), sI);
                    else if (fwd) add(t, 1.0, rb.st({KC, (int16_t)p, -1}), s_cd[site_of(q)]);    // a+p^L a+q^C
                    else add(t, 1.0, rb.st({KC, (int16_t)q, -1}), s_cd[site_of(p)]);             // a+p^C a+q^R
                    break;
                case KB:
                    if (inC(p) && inC(q)) addS(t, 1.0, Iref, local_mul(cd[site_of(p)], an[site_of(q)]));
                    else if (!inC(p) && !inC(q)) add(t, 1.0, rb.st(key), sI);
                    else if (fwd) {
                        if (!inC(p)) add(t, 1.0, rb.st({KC, (int16_t)p, -1}), s_an[site_of(q)]);  // a+p^L a_s^C
                        else add(t, -1.0, rb.st({KC, (int16_t)q, -1}, true), s_cd[site_of(p)]);   // -a_s^L a+p^C
                    } else {
                        if (inC(p)) add(t, 1.0, rb.st({KC, (int16_t)q, -1}, true), s_cd[site_of(p)]);  // a+p^C a_s^R
                        else add(t, -1.0, rb.st({KC, (int16_t)p, -1}), s_an[site_of(q)]);          // -a_s^C a+p^R
                    }
                    break;
                case KS: {
                    add(t, 1.0, rb.st(key), sI);
                    addS(t, 1.0, Iref, SC_full(p));
                    // sum_{q in big} a+q P^C_pq  (forward)  /  sum_{q in big} P^C_pq a+q (backward)
                    OpRef x = rb.lin(CB, [&](int i) { return I.w(p, P_(CB, i), c0, c0 + 1); });
                    add(t, 1.0, x, S(aa));
                    // sum_{q in C} P^big_pq a+q^C
                    for (int a = 0; a < 2; ++a) {
                        int qq = co[a];
                        OpRef xp = rb.lin(ABt, [&](int i) { return I.w(p, qq, P_(ABt, i), Q_(ABt, i)); });
                        add(t, 1.0, xp, s_cd[a]);
                    }
                    // sum_{r in C} Q^big_pr a_r^C
                    for (int a = 0; a < 2; ++a) {
                        int r = co[a];
                        OpRef xq = rb.lin(BB, [&](int i) { return I.w(p, P_(BB, i), r, Q_(BB, i)); });
                        add(t, 1.0, xq, s_an[a]);
                    }
                    // sum_{s in big} a_s Q^C_ps, Q^C_ps = sum_{q,r in C} w_pqsr a+q a_r
                    for (int a = 0; a < 2; ++a)
                        for (int b = 0; b < 2; ++b) {
                            int qq = co[a], r = co[b];
                            OpRef xs = rb.lin(CBt, [&](int i) { return I.w(p, qq, P_(CBt, i), r); });
                            add(t, 1.0, xs, S(local_mul(cd[a], an[b])));
                        }
                    break;
                }
                case KH: {
                    add(t, 1.0, rb.st(key), sI);
                    addS(t, 1.0, Iref, HC);
                    // big-block orbital p with S^C_p (+ h.c.), sign of the reordering
                    for (auto& e : SCel) {
                        auto fc = e.second;
                        OpRef x = rb.lin(CB, [&](int i) { return fc(P_(CB, i)); });
                        if (fwd) {  // a+p^L S^C_p - a_p^L (S^C_p)^T
                            add(t, 1.0, x, e.first);
                            add(t, -1.0, flip(x), P.site.transpose(e.first));
                        } else {    // a+p^R S^C_p = -S^C_p a+p^R ; h.c. = (S^C_p)^T a_p^R
                            add(t, -1.0, x, e.first);
                            add(t, 1.0, flip(x), P.site.transpose(e.first));
                        }
                    }
                    // site orbital p with S^big_p (+ h.c.)
                    for (int a = 0; a < 2; ++a) {
                        int pp = co[a];
                        OpKey ks{KS, (int16_t)pp, -1};
                        if (fwd) {  // a+p^C S^L_p = -S^L_p a+p^C ; h.c. = (S^L_p)^T a_p^C
                            add(t, -1.0, rb.st(ks), s_cd[a]);
                            add(t, 1.0, rb.st(ks, true), s_an[a]);
                        } else {    // a+p^C S^R_p ; h.c. = -a_p^C (S^R_p)^T
                            add(t, 1.0, rb.st(ks), s_cd[a]);
                            add(t, -1.0, rb.st(ks, true), s_an[a]);
                        }
                    }
                    // normal operators on the site: A^C P^big + h.c., B^C Q^big
                    OpRef xp = rb.lin(ABt, [&](int i) { return I.w(c0, c0 + 1, P_(ABt, i), Q_(ABt, i)); });
                    add(t, 1.0, xp, S(AC));
                    add(t, 1.0, flip(xp), S(local_T(AC)));
                    for (int a = 0; a < 2; ++a)
                        for (int b = 0; b < 2; ++b) {
                            int pp = co[a], ss = co[b];
                            OpRef xq = rb.lin(BB, [&](int i) { return I.w(pp, P_(BB, i), ss, Q_(BB, i)); });
                            add(t, 1.0, xq, S(local_mul(cd[a], an[b])));
                        }
                    break;
                }
                default: break;
            }
            P.targets.push_back(std::move(t));
        }
    }
}

}  // namespace dmrg

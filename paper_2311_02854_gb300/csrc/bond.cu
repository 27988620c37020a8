// Environments and the current bond: vacuum blocks, renormalisation
// (Eq. Renorm / Eqs. renorm12-renormFinal), the bond's intermediates (the
// "intermediates" step of Sec. 2.2) and the sigma / diag(H_eff) work lists
// (Eqs. sigmablk56-sigmablk).
#include <algorithm>
#include <cmath>

#include "bond.h"

namespace dmrg {

namespace {

// Buffer ids of the BufTable used by every work list.
enum : int8_t { BUF_L = 0, BUF_R = 1, BUF_INT = 2, BUF_PSI = 3, BUF_SCR = 4, BUF_ID = 5, BUF_OUT = 6, BUF_W = 7 };

struct OpLookup {
    bool ok = false;
    int j = -1;   // bra sector
    View v;       // view of the effective operator block (d_j x d_i)
};

}  // namespace

// Lookup of an operator reference acting on ket sector i of `lay`.
// Stored rows live in buffer `store_buf`, intermediates in BUF_INT.
static OpLookup lookup(const BlockLayout& lay, const Interms& im, const OpRef& r, int i, int8_t store_buf) {
    OpLookup o;
    if (r.src == SRC_I) {
        o.ok = true;
        o.j = i;
        o.v.ident = true;
        return o;
    }
    const Family* f;
    int64_t rowbase;
    int8_t buf;
    if (r.src == SRC_STORE) {
        f = &lay.fams[r.fam];
        rowbase = f->base + (int64_t)r.row * f->stride;
        buf = store_buf;
    } else {
        const IntermFamily& IF = im.fams[r.fam];
        f = &lay.fams[IF.src_fam];
        rowbase = IF.base + (int64_t)r.row * f->stride;
        buf = BUF_INT;
    }
    const Basis& b = lay.basis;
    if (!r.tr) {
        int pr = f->pair_of_ket[i];
        if (pr < 0) return o;
        o.j = f->bra[pr];
        o.v.buf = buf;
        o.v.off = rowbase + f->off[pr];
        o.v.ld = f->ld[pr];
        o.v.tr = false;
    } else {
        int j = b.find(b.qn[i] - f->dq);
        if (j < 0) return o;
        int pr = f->pair_of_ket[j];
        if (pr < 0) return o;
        o.j = j;
        o.v.buf = buf;
        o.v.off = rowbase + f->off[pr];
        o.v.ld = f->ld[pr];
        o.v.tr = true;
    }
    o.ok = true;
    return o;
}

static int ref_parity(const BlockLayout& lay, const Interms& im, const OpRef& r) {
    if (r.src == SRC_I) return 0;
    if (r.src == SRC_STORE) return kind_parity(lay.fams[r.fam].kind);
    return kind_parity(lay.fams[im.fams[r.fam].src_fam].kind);
}

// ---------------------------------------------------------------------------
// Intermediates: Int[rows x nnz] = W[rows x nops] * Family[nops x nnz]
// ---------------------------------------------------------------------------

void form_interms(Plan& P, Interms& im, const Block* blocks[2], double*& d_int, int64_t& n_int,
                  double& flops) {
    int64_t total = 0, wtot = 0;
    for (auto& IF : im.fams) {
        const Family& f = blocks[IF.owner]->lay.fams[IF.src_fam];
        IF.base = total;
        total += (int64_t)IF.rows.size() * f.stride;
        wtot += (int64_t)IF.rows.size() * f.nops();
    }
    P.free(d_int, n_int);
    n_int = total;
    d_int = P.alloc(std::max<int64_t>(total, 1));
    flops = 0.0;
    if (im.fams.empty()) return;
    std::vector<double> W(wtot, 0.0);
    WorkList wl;
    int64_t woff = 0;
    for (auto& IF : im.fams) {
        const Family& f = blocks[IF.owner]->lay.fams[IF.src_fam];
        const int nr = (int)IF.rows.size(), no = f.nops();
        for (int r = 0; r < nr; ++r)
            for (auto& rc : IF.rows[r]) W[woff + (int64_t)r * no + rc.first] += rc.second;
        Seg s{};
        s.a_off = woff;
        s.b_off = f.base;
        s.k = no;
        s.lda = no;
        s.ldb = (int)f.stride;
        DMRG_REQUIRE(f.stride < (1LL << 31), DMRG_EINVAL, "operator family too large");
        s.a_buf = BUF_W;
        s.b_buf = (uint8_t)IF.owner;  // BUF_L or BUF_R
        s.alpha = 1.0;
        wl.add_block(IF.base, BUF_INT, nr, (int)f.nnz, (int)f.stride, {s}, TILE_STORE);
        woff += (int64_t)nr * no;
    }
    flops = wl.flops;
    if (wtot > P.n_wcoef) {
        P.free(P.d_wcoef, P.n_wcoef);
        P.n_wcoef = wtot;
        P.d_wcoef = P.alloc(wtot);
    }
    DMRG_CHECK_CUDA(cudaMemcpyAsync(P.d_wcoef, W.data(), wtot * 8, cudaMemcpyHostToDevice, P.stream));
    wl.upload(P.stream);
    BufTable bt{};
    bt.p[BUF_L] = blocks[0] ? blocks[0]->d : nullptr;
    bt.p[BUF_R] = blocks[1] ? blocks[1]->d : nullptr;
    bt.p[BUF_INT] = d_int;
    bt.p[BUF_W] = P.d_wcoef;
    launch_seg_gemm_f64(wl, bt, 1, P.stream);
    DMRG_CHECK_CUDA(cudaStreamSynchronize(P.stream));
    wl.release();
}

void ensure_ident(Plan& P, int n) {
    if (n <= P.ident_n) return;
    P.free(P.d_ident, (int64_t)P.ident_n * P.ident_n);
    P.ident_n = std::max(n, 64);
    P.d_ident = P.alloc((int64_t)P.ident_n * P.ident_n);
    dev_identity(P.d_ident, P.ident_n, P.stream);
}

void ensure_scratch(Plan& P, int64_t n) {
    if (n <= P.n_scratch) return;
    P.free(P.d_scratch, P.n_scratch);
    P.n_scratch = n;
    P.d_scratch = P.alloc(n);
}

int64_t scratch_cap(const Plan& P) {
    int64_t cap = P.opt.scratch_bytes > 0 ? P.opt.scratch_bytes / 8 : 0;
    if (cap <= 0) cap = std::max<int64_t>((int64_t)1 << 26, P.budget / 8 / 16);  // >= 512 MiB
    return cap;
}

// ---------------------------------------------------------------------------
// Blocks
// ---------------------------------------------------------------------------

std::unique_ptr<Block> make_vacuum(Plan& P, bool right_end) {
    auto B = std::make_unique<Block>();
    Basis b;
    b.add(QN(0, 0), 1);
    int lo = right_end ? P.n_so : 0;
    B->lay.build(b, lo, lo, P.n_so);
    B->n = std::max<int64_t>(B->lay.total, 1);
    B->d = P.alloc(B->n);
    dev_fill(B->d, 0.0, B->n, P.stream);
    return B;
}

Basis bond_basis(const Plan& P, int b, bool right_side) {
    Basis bs;
    for (auto& s : P.mps.bonds[b]) {
        QN lab(s[0], s[1]);
        bs.add(right_side ? P.tot - lab : lab, s[2]);
    }
    return bs;
}

// Packed device copy of site tensor A[k]; key -> (offset, d_l, d_r)
struct SiteDev {
    double* d = nullptr;
    int64_t n = 0;
    std::map<std::array<int, 3>, int64_t> off;
};

static SiteDev upload_site(Plan& P, int k) {
    SiteDev S;
    int64_t tot = 0;
    for (auto& kv : P.mps.sites[k]) {
        S.off[kv.first] = tot;
        tot += (int64_t)kv.second.size();
    }
    S.n = std::max<int64_t>(tot, 1);
    S.d = P.alloc(S.n);
    std::vector<double> host(S.n, 0.0);
    for (auto& kv : P.mps.sites[k])
        std::copy(kv.second.begin(), kv.second.end(), host.begin() + S.off[kv.first]);
    DMRG_CHECK_CUDA(cudaMemcpyAsync(S.d, host.data(), S.n * 8, cudaMemcpyHostToDevice, P.stream));
    DMRG_CHECK_CUDA(cudaStreamSynchronize(P.stream));
    return S;
}

// Grow block X by site m (forward: X = sites 1..m-1 -> sites 1..m) or
// (backward: X = sites m+1..K -> sites m..K) with the site tensor A[m].
std::unique_ptr<Block> renormalise(Plan& P, const Block& X, int m, bool forward) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, P.stream);
    auto out = std::make_unique<Block>();
    const int k0 = m - 1;
    if (forward) out->lay.build(bond_basis(P, m, false), 0, 2 * m, P.n_so);
    else out->lay.build(bond_basis(P, m - 1, true), 2 * (m - 1), P.n_so, P.n_so);
    const BlockLayout& XL = X.lay;
    const BlockLayout& OL = out->lay;
    RenormPlan rp;
    build_renorm_terms(P.I, XL, OL, k0, forward, rp);
    // intermediates on X
    const Block* blocks[2] = {&X, nullptr};
    double* d_int = nullptr;
    int64_t n_int = 0;
    double fl_int = 0.0;
    form_interms(P, rp.interms, blocks, d_int, n_int, fl_int);
    SiteDev A = upload_site(P, m);
    out->n = std::max<int64_t>(OL.total, 1);
    out->d = P.alloc(out->n);
    DMRG_CHECK_CUDA(cudaMemsetAsync(out->d, 0, out->n * 8, P.stream));

    ProductList pl;
    std::map<std::pair<int, int>, int> outidx;  // (target, pair) -> out block
    auto site_key = [&](int il, int n, int ir) {
        auto it = A.off.find({il, n, ir});
        return it == A.off.end() ? (int64_t)-1 : it->second;
    };
    // index A blocks by ket component
    std::vector<std::array<int, 3>> keys;
    for (auto& kv : P.mps.sites[m]) keys.push_back(kv.first);
    const auto& bl = P.mps.bonds[m - 1];
    const auto& br = P.mps.bonds[m];
    // bra lookup: forward (jl, c') -> jr ; backward (n', jr) -> jl
    std::map<std::pair<int, int>, int> fwd_bra, bwd_bra;
    for (auto& kk : keys) {
        fwd_bra[{kk[0], kk[1]}] = kk[2];
        bwd_bra[{kk[1], kk[2]}] = kk[0];
    }
    for (int t = 0; t < (int)rp.targets.size(); ++t) {
        const RenormTarget& T = rp.targets[t];
        auto fr = OL.find(T.key);
        const Family& of = OL.fams[fr.first];
        const int64_t obase = of.base + (int64_t)fr.second * of.stride;
        for (const Term2& term : T.terms) {
            const LocalOp& M = rp.site.ops[term.site];
            const int parX = ref_parity(XL, rp.interms, term.X);
            for (auto& kk : keys) {
                const int il = kk[0], n = kk[1], ir = kk[2];
                if (forward) {
                    // ket component (il, n) of X.C -> new sector ir; X acts on il
                    OpLookup ox = lookup(XL, rp.interms, term.X, il, BUF_L);
                    if (!ox.ok) continue;
                    const int jl = ox.j;
                    for (int c2 = 0; c2 < 4; ++c2) {
                        double mv = M.at(c2, n);
                        if (mv == 0.0) continue;
                        auto bj = fwd_bra.find({jl, c2});
                        if (bj == fwd_bra.end()) continue;
                        const int jr = bj->second;
                        int pr = of.pair_of_ket[ir];
                        if (pr < 0 || of.bra[pr] != jr) continue;
                        const int dl = bl[il][2], djl = bl[jl][2], dr = br[ir][2], djr = br[jr][2];
                        double zeta = (M.parity && (XL.basis.qn[il].n & 1)) ? -1.0 : 1.0;
                        auto key = std::make_pair(t, pr);
                        auto oi = outidx.find(key);
                        int o;
                        if (oi == outidx.end()) {
                            o = (int)pl.outs.size();
                            outidx[key] = o;
                            pl.outs.push_back({BUF_R, obase + of.off[pr], djr, dr, of.ld[pr]});
                        } else {
                            o = oi->second;
                        }
                        Contrib c;
                        c.out = o;
                        c.P.buf = BUF_PSI;
                        c.P.off = site_key(jl, c2, jr);
                        c.P.ld = djr;
                        c.P.tr = true;  // A(jl,c2,jr)^T : djr x djl
                        c.Q = ox.v;     // X_eff : djl x dl
                        c.R.buf = BUF_PSI;
                        c.R.off = site_key(il, n, ir);
                        c.R.ld = dr;    // A(il,n,ir) : dl x dr
                        c.m = djr;
                        c.k1 = djl;
                        c.k2 = dl;
                        c.n = dr;
                        c.alpha = term.c * zeta * mv;
                        pl.cs.push_back(c);
                    }
                } else {
                    // ket component (n, ir) of C.X -> new sector il; X acts on ir
                    OpLookup ox = lookup(XL, rp.interms, term.X, ir, BUF_L);
                    if (!ox.ok) continue;
                    const int jr = ox.j;
                    for (int n2 = 0; n2 < 4; ++n2) {
                        double mv = M.at(n2, n);
                        if (mv == 0.0) continue;
                        auto bj = bwd_bra.find({n2, jr});
                        if (bj == bwd_bra.end()) continue;
                        const int jl = bj->second;
                        int pr = of.pair_of_ket[il];
                        if (pr < 0 || of.bra[pr] != jl) continue;
                        const int dl = bl[il][2], djl = bl[jl][2], dr = br[ir][2], djr = br[jr][2];
                        double zeta = (parX && (kSiteQN[n].n & 1)) ? -1.0 : 1.0;
                        auto key = std::make_pair(t, pr);
                        auto oi = outidx.find(key);
                        int o;
                        if (oi == outidx.end()) {
                            o = (int)pl.outs.size();
                            outidx[key] = o;
                            pl.outs.push_back({BUF_R, obase + of.off[pr], djl, dl, of.ld[pr]});
                        } else {
                            o = oi->second;
                        }
                        Contrib c;
                        c.out = o;
                        c.P.buf = BUF_PSI;
                        c.P.off = site_key(jl, n2, jr);
                        c.P.ld = djr;   // A(jl,n2,jr) : djl x djr
                        c.Q = ox.v;     // X_eff : djr x dr
                        c.R.buf = BUF_PSI;
                        c.R.off = site_key(il, n, ir);
                        c.R.ld = dr;
                        c.R.tr = true;  // A(il,n,ir)^T : dr x dl
                        c.m = djl;
                        c.k1 = djr;
                        c.k2 = dr;
                        c.n = dl;
                        c.alpha = term.c * zeta * mv;
                        pl.cs.push_back(c);
                    }
                }
            }
        }
    }
    int maxd = std::max({XL.basis.dmax(), OL.basis.dmax(), 1});
    ensure_ident(P, maxd);
    const int64_t cap = scratch_cap(P);
    pl.lower(BUF_SCR, BUF_ID, P.ident_n, cap, 1 << 14);
    ensure_scratch(P, std::max<int64_t>(pl.scratch_elems, 1));
    pl.upload(P.stream);
    BufTable bt{};
    bt.p[BUF_L] = X.d;
    bt.p[BUF_R] = out->d;
    bt.p[BUF_INT] = d_int;
    bt.p[BUF_PSI] = A.d;
    bt.p[BUF_SCR] = P.d_scratch;
    bt.p[BUF_ID] = P.d_ident;
    pl.run(bt, 1, P.stream);
    cudaEventRecord(e1, P.stream);
    DMRG_CHECK_CUDA(cudaStreamSynchronize(P.stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    P.stats.ms_renorm += ms;
    P.stats.renorm_flops_last = pl.flops + fl_int;
    pl.release();
    P.free(d_int, n_int);
    P.free(A.d, A.n);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return out;
}

// ---------------------------------------------------------------------------
// Current bond
// ---------------------------------------------------------------------------

void ensure_env(Plan& P, int k) {
    const int K = P.K;
    // left[k-1]
    if (!P.left[0]) P.left[0] = make_vacuum(P, false);
    int m = k - 1;
    int have = m;
    while (have > 0 && !P.left[have]) --have;
    for (int j = have + 1; j <= m; ++j) {
        P.left[j] = renormalise(P, *P.left[j - 1], j, true);
        if (!P.opt.keep_envs && j - 1 >= 1) {
            P.free(P.left[j - 1]->d, P.left[j - 1]->n);
            P.left[j - 1].reset();
        }
    }
    if (!P.right[K]) P.right[K] = make_vacuum(P, true);
    int mr = k + 1;
    int haver = mr;
    while (haver < K && !P.right[haver]) ++haver;
    for (int j = haver - 1; j >= mr; --j) {
        P.right[j] = renormalise(P, *P.right[j + 1], j + 1, false);
        if (!P.opt.keep_envs && j + 1 <= K - 1) {
            P.free(P.right[j + 1]->d, P.right[j + 1]->n);
            P.right[j + 1].reset();
        }
    }
}

void build_layout(Plan& P, int k) {
    P.layout.clear();
    P.sector_of.clear();
    const auto& bl = P.mps.bonds[k - 1];
    const auto& br = P.mps.bonds[k + 1];
    std::map<std::pair<int, int>, int> ridx;
    for (int i = 0; i < (int)br.size(); ++i) ridx[{br[i][0], br[i][1]}] = i;
    int64_t off = 0;
    for (int il = 0; il < (int)bl.size(); ++il)
        for (int y = 0; y < 16; ++y) {
            QN q = QN(bl[il][0], bl[il][1]) + kSiteQN[y / 4] + kSiteQN[y % 4];
            auto it = ridx.find({q.n, q.s});
            if (it == ridx.end()) continue;
            Plan::Sector s{il, y, it->second, off, bl[il][2], br[it->second][2]};
            P.sector_of[{il, y}] = (int)P.layout.size();
            P.layout.push_back(s);
            off += (int64_t)s.dl * s.dr;
        }
    P.dim = off;
}

void set_bond(Plan& P, int k) {
    DMRG_REQUIRE(k >= 1 && k <= P.K - 1, DMRG_EINVAL, "bond index out of range");
    DMRG_REQUIRE(k == P.mps.center, DMRG_EINVAL,
                 "bond " + std::to_string(k) + " is not the MPS centre " + std::to_string(P.mps.center));
    ensure_env(P, k);
    const Block& L = *P.left[k - 1];
    const Block& R = *P.right[k + 1];
    build_layout(P, k);
    build_sigma_terms(P.I, L.lay, R.lay, k, P.sp);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, P.stream);
    const Block* blocks[2] = {&L, &R};
    double fl = 0.0;
    form_interms(P, P.sp.interms, blocks, P.d_interm, P.n_interm, fl);
    cudaEventRecord(e1, P.stream);
    DMRG_CHECK_CUDA(cudaStreamSynchronize(P.stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    P.stats.ms_interm += ms;
    P.stats.interm_flops = fl;
    P.stats.interm_bytes = P.n_interm * 8;
    P.stats.store_bytes = (L.n + R.n) * 8;

    // sigma contributions
    ProductList& pl = P.sigma_pl;
    pl.clear();
    for (const Plan::Sector& s : P.layout) {
        pl.outs.push_back({BUF_OUT, s.off, s.dl, s.dr, s.dr});
    }
    const LocalOps& Y = P.sp.y;
    int64_t nitems = 0;
    for (const Term3& t : P.sp.terms) {
        const LocalOp& M = Y.ops[t.y];
        const int pR = ref_parity(R.lay, P.sp.interms, t.R);
        for (const Plan::Sector& s : P.layout) {
            OpLookup ol = lookup(L.lay, P.sp.interms, t.L, s.il, BUF_L);
            if (!ol.ok) continue;
            OpLookup orr = lookup(R.lay, P.sp.interms, t.R, s.ir, BUF_R);
            if (!orr.ok) continue;
            const int nl = L.lay.basis.qn[s.il].n;
            const int ny = kSiteQN[s.y / 4].n + kSiteQN[s.y % 4].n;
            for (int y2 = 0; y2 < 16; ++y2) {
                double mv = M.at(y2, s.y);
                if (mv == 0.0) continue;
                auto it = P.sector_of.find({ol.j, y2});
                DMRG_REQUIRE(it != P.sector_of.end() || true, DMRG_EINVAL, "");
                if (it == P.sector_of.end()) continue;
                const Plan::Sector& o = P.layout[it->second];
                DMRG_REQUIRE(o.ir == orr.j, DMRG_EINVAL, "sigma term breaks the symmetry");
                int e = M.parity * nl + pR * (nl + ny);
                double zeta = (e & 1) ? -1.0 : 1.0;
                Contrib c;
                c.out = it->second;
                c.P = ol.v;  // O^L_eff : d_jl x d_il
                c.Q.buf = BUF_PSI;
                c.Q.off = s.off;
                c.Q.ld = s.dr;  // Psi_s : d_il x d_ir
                c.R = orr.v.T();  // (O^R_eff)^T : d_ir x d_jr
                c.R.ident = orr.v.ident;
                c.m = o.dl;
                c.k1 = s.dl;
                c.k2 = s.dr;
                c.n = o.dr;
                c.alpha = t.c * zeta * mv;
                pl.cs.push_back(c);
                ++nitems;
            }
        }
    }
    int maxd = std::max({L.lay.basis.dmax(), R.lay.basis.dmax(), 1});
    ensure_ident(P, maxd);
    pl.lower(BUF_SCR, BUF_ID, P.ident_n, scratch_cap(P), 1 << 14);
    ensure_scratch(P, std::max<int64_t>(pl.scratch_elems, 1));
    pl.upload(P.stream);
    P.stats.n_terms = (int64_t)P.sp.terms.size();
    P.stats.n_items = nitems;
    P.stats.sigma_flops = pl.flops;

    // diag(H_eff): terms whose three factors all conserve the quantum numbers
    ProductList& hl = P.hdiag_pl;
    hl.clear();
    {
        WorkList w;
        std::vector<std::vector<Seg>> per(P.layout.size());
        for (const Term3& t : P.sp.terms) {
            const LocalOp& M = Y.ops[t.y];
            if (M.dq != QN(0, 0)) continue;
            const int pR = ref_parity(R.lay, P.sp.interms, t.R);
            for (size_t si = 0; si < P.layout.size(); ++si) {
                const Plan::Sector& s = P.layout[si];
                double mv = M.at(s.y, s.y);
                if (mv == 0.0) continue;
                OpLookup ol = lookup(L.lay, P.sp.interms, t.L, s.il, BUF_L);
                if (!ol.ok || ol.j != s.il) continue;
                OpLookup orr = lookup(R.lay, P.sp.interms, t.R, s.ir, BUF_R);
                if (!orr.ok || orr.j != s.ir) continue;
                const int nl = L.lay.basis.qn[s.il].n;
                const int ny = kSiteQN[s.y / 4].n + kSiteQN[s.y % 4].n;
                int e = M.parity * nl + pR * (nl + ny);
                double zeta = (e & 1) ? -1.0 : 1.0;
                View a = ol.v, b = orr.v;
                if (a.ident) {
                    a.buf = BUF_ID;
                    a.off = 0;
                    a.ld = P.ident_n;
                }
                if (b.ident) {
                    b.buf = BUF_ID;
                    b.off = 0;
                    b.ld = P.ident_n;
                }
                // diagonal as a (d x 1) column / (1 x d) row: stride ld + 1
                Seg sg{};
                sg.a_off = a.off;
                sg.lda = a.ld + 1;
                sg.a_tr = 0;
                sg.a_buf = (uint8_t)a.buf;
                sg.b_off = b.off;
                sg.ldb = b.ld + 1;
                sg.b_tr = 1;
                sg.b_buf = (uint8_t)b.buf;
                sg.k = 1;
                sg.alpha = t.c * zeta * mv;
                per[si].push_back(sg);
            }
        }
        for (size_t si = 0; si < P.layout.size(); ++si) {
            const Plan::Sector& s = P.layout[si];
            w.add_block(s.off, BUF_OUT, s.dl, s.dr, s.dr, per[si], TILE_STORE);
        }
        hl.chunks.emplace_back(WorkList(), std::move(w));
        hl.upload(P.stream);
    }
    P.bond = k;
    DMRG_CHECK_CUDA(cudaStreamSynchronize(P.stream));
}

BufTable bond_buffers(Plan& P, const double* psi, double* out) {
    BufTable bt{};
    bt.p[BUF_L] = P.left[P.bond - 1]->d;
    bt.p[BUF_R] = P.right[P.bond + 1]->d;
    bt.p[BUF_INT] = P.d_interm;
    bt.p[BUF_PSI] = const_cast<double*>(psi);
    bt.p[BUF_SCR] = P.d_scratch;
    bt.p[BUF_ID] = P.d_ident;
    bt.p[BUF_OUT] = out;
    bt.vstride[BUF_PSI] = P.dim;
    bt.vstride[BUF_OUT] = P.dim;
    bt.vstride[BUF_SCR] = P.sigma_pl.scratch_elems;
    return bt;
}

void sigma(Plan& P, const double* psi, double* out, int nvec, cudaStream_t st) {
    DMRG_REQUIRE(P.bond > 0, DMRG_EINVAL, "no current bond (call dmrg_set_bond)");
    DMRG_REQUIRE(nvec >= 1, DMRG_EINVAL, "nvec must be >= 1");
    // scratch is per vector: run in groups that fit
    int64_t per = std::max<int64_t>(P.sigma_pl.scratch_elems, 1);
    int group = (int)std::max<int64_t>(1, std::min<int64_t>(nvec, P.n_scratch / per));
    for (int v0 = 0; v0 < nvec; v0 += group) {
        int nv = std::min(group, nvec - v0);
        DMRG_CHECK_CUDA(cudaMemsetAsync(out + (int64_t)v0 * P.dim, 0, (size_t)nv * P.dim * 8, st));
        if (nv > 1) ensure_scratch(P, per * nv);
        BufTable bt = bond_buffers(P, psi + (int64_t)v0 * P.dim, out + (int64_t)v0 * P.dim);
        bt.vstride[BUF_SCR] = per;
        P.sigma_pl.run(bt, nv, st);
    }
    P.stats.sigma_calls += nvec;
}

void hdiag(Plan& P, double* out, cudaStream_t st) {
    DMRG_REQUIRE(P.bond > 0, DMRG_EINVAL, "no current bond (call dmrg_set_bond)");
    BufTable bt = bond_buffers(P, nullptr, out);
    P.hdiag_pl.run(bt, 1, st);
}

}  // namespace dmrg

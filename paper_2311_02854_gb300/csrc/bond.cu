// Environments and the current bond: vacuum blocks, renormalisation
// (Eq. Renorm / Eqs. renorm12-renormFinal), the bond's intermediates (the
// "intermediates" step of Sec. 2.2) and the sigma / diag(H_eff) work lists
// (Eqs. sigmablk56-sigmablk).  Two engines share the planning: FP64 (SIMT
// kernel, 64x64 tiles) and the tcgen05 engine on bf16 pieces (mixed precision).
#include <algorithm>
#include <chrono>
#include <cmath>

#include "bond.h"

namespace dmrg {

namespace {

// Buffer ids of the tables used by every work list.
enum : int8_t { BUF_L = 0, BUF_R = 1, BUF_INT = 2, BUF_PSI = 3, BUF_SCR = 4, BUF_ID = 5, BUF_OUT = 6, BUF_W = 7 };

constexpr int64_t kChunkF64 = 1 << 14;  // K-depth per accumulation pass (FP64 engine)
// Tensor cores: K-depth one output tile accumulates in FP32 tensor memory
// before it is added (atomically) into an FP64 result.  The error of a chain
// grows linearly with its depth (about 6e-6 relative at 1024 on sigma-like
// sums), so chains are kept short; the operator store (renormalisation,
// intermediates), whose error every later bond inherits, uses the shortest.
constexpr int64_t kChunkTC = 256;        // renormalisation and intermediates
constexpr int64_t kChunkSigmaTC = 1024;  // sigma, two pieces
constexpr int64_t kChunkSigmaX6 = 256;   // sigma, three pieces

struct OpLookup {
    bool ok = false;
    int j = -1;  // bra sector
    View v;      // view of the effective operator block (d_j x d_i)
};

// Lookup of an operator reference acting on ket sector i of `lay`.
// Stored rows live in buffer `store_buf`, intermediates in BUF_INT.
OpLookup lookup(const BlockLayout& lay, const Interms& im, const OpRef& r, int i, int8_t store_buf) {
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
    int nrows;
    if (r.src == SRC_STORE) {
        f = &lay.fams[r.fam];
        rowbase = f->base + (int64_t)r.row * f->stride;
        buf = store_buf;
        nrows = f->nops();
    } else {
        const IntermFamily& IF = im.fams[r.fam];
        f = &lay.fams[IF.src_fam];
        rowbase = IF.base + (int64_t)r.row * f->stride;
        buf = BUF_INT;
        nrows = (int)IF.rows.size();
    }
    o.v.z = r.row;
    o.v.nz = nrows;
    o.v.zstride = f->stride;
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

int ref_parity(const BlockLayout& lay, const Interms& im, const OpRef& r) {
    if (r.src == SRC_I) return 0;
    if (r.src == SRC_STORE) return kind_parity(lay.fams[r.fam].kind);
    return kind_parity(lay.fams[im.fams[r.fam].src_fam].kind);
}

double host_ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

void ensure_counter(Plan& P) {
    if (!P.d_ctr) {
        DMRG_CHECK_CUDA(cudaMalloc(&P.d_ctr, 2 * sizeof(int)));
        DMRG_CHECK_CUDA(cudaMemset(P.d_ctr, 0, 2 * sizeof(int)));
    }
}

TcBufs tc_base(Plan& P) {
    ensure_counter(P);
    TcBufs tb{};
    tb.counter = P.d_ctr;
    tb.err = P.d_ctr + 1;
    return tb;
}

// piece pointers of buffer b (n elements per piece)
void set_pieces(const Plan& P, TcBufs& tb, int b, const __nv_bfloat16* hi, const __nv_bfloat16* lo, int64_t n) {
    tb.hi[b] = hi;
    tb.lo[b] = lo;
    tb.pstride[b] = P.nsplit == 3 ? n : 0;
}
void set_out_pieces(const Plan& P, TcBufs& tb, int b, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t n) {
    tb.out[b] = hi;
    tb.out_lo[b] = lo;
    tb.out_pstride[b] = P.nsplit == 3 ? n : 0;
}

// bf16 pieces of the padded wavefunction copy for n elements (all vectors of a launch)
void ensure_psi_pieces(Plan& P, int64_t n) {
    if (n <= P.n_ppc) return;
    P.free_bf16(P.ps_hi, P.n_ppc);
    P.free_lo(P.ps_lo, P.n_ppc);
    P.n_ppc = n;
    P.ps_hi = P.alloc_bf16(n);
    P.ps_lo = P.alloc_lo(n);
}

// Buffers of the mixed sigma at bond k (out: FP64 result of vector 0)
TcBufs sigma_bufs(Plan& P, int k, double* out) {
    DMRG_REQUIRE(k >= 1 && k <= P.K - 1 && P.left[k - 1] && P.right[k + 1], DMRG_EINVAL,
                 "sigma buffers requested without the bond's environments");
    const Block& L = *P.left[k - 1];
    const Block& R = *P.right[k + 1];
    const int64_t per = std::max<int64_t>(P.sigma_tc.scratch_elems, 8);
    TcBufs tb = tc_base(P);
    set_pieces(P, tb, BUF_L, L.h, L.l, L.n);
    set_pieces(P, tb, BUF_R, R.h, R.l, R.n);
    set_pieces(P, tb, BUF_INT, P.interm.h, P.interm.l, P.interm.n);
    set_pieces(P, tb, BUF_PSI, P.ps_hi, P.ps_lo, P.n_ppc);
    tb.vstride[BUF_PSI] = P.dim_pad;
    set_pieces(P, tb, BUF_SCR, P.s_hi, P.s_lo, P.n_spc);
    tb.vstride[BUF_SCR] = per;
    set_pieces(P, tb, BUF_ID, P.id_hi, P.id_lo, (int64_t)P.id_n * P.id_n);
    tb.out[BUF_OUT] = out;
    tb.out_vstride[BUF_OUT] = P.dim;
    set_out_pieces(P, tb, BUF_SCR, P.s_hi, P.s_lo, P.n_spc);
    tb.out_vstride[BUF_SCR] = per;
    return tb;
}

// ---------------------------------------------------------------------------
// Tile-shape autotuner of the mixed sigma
// ---------------------------------------------------------------------------

// Key of the bond's sector-size histogram, coarse enough that the bonds of one
// region of a sweep share it: the size classes (limits 16 ... 384) of the
// largest row and column sector, the number of sectors, of psi elements and
// of terms on a log2 scale, the piece count and the vectors per launch.
uint64_t sector_histogram_key(const Plan& P, int G) {
    static const int cuts[7] = {16, 32, 64, 128, 192, 256, 384};
    auto cls = [&](int d) {
        int c = 0;
        while (c < 7 && d > cuts[c]) ++c;
        return c;
    };
    auto lg = [](int64_t x) {
        int l = 0;
        while (((int64_t)1 << l) <= x) ++l;
        return l;
    };
    int dl = 0, dr = 0;
    for (const Plan::Sector& s : P.layout) {
        dl = std::max(dl, s.dl);
        dr = std::max(dr, s.dr);
    }
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t x) {
        h ^= x;
        h *= 1099511628211ull;
    };
    mix((uint64_t)P.nsplit);
    mix((uint64_t)G);
    mix((uint64_t)cls(dl));
    mix((uint64_t)cls(dr));
    mix((uint64_t)lg((int64_t)P.layout.size()));
    mix((uint64_t)lg(P.dim));
    mix((uint64_t)lg((int64_t)P.sp.terms.size()));
    return h;
}

struct SigmaShape {
    int tn;
    int64_t kchunk;
};

// Times the candidate shapes (tile width 128 / 64, phase-2 K-chunk kmax /
// kmax/2) on a sample of the bond's work list: every 8th (16th) output block
// with all of its products, lowered exactly as the full list would be.  Each
// candidate runs once to warm up and once timed (CUDA events on the plan's
// stream); the fastest wins, the default (128, kmax) unless another is 2 %
// faster.
SigmaShape tune_sigma_shape(Plan& P, int k, const ProductList& tl, int64_t cap, int64_t kmax, const int64_t* vs,
                            int G) {
    const uint64_t key = sector_histogram_key(P, G);
    auto f = P.tune_cache.find(key);
    if (f != P.tune_cache.end()) {
        ++P.stats.tune_hits;
        return {f->second.first, f->second.second};
    }
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t khalf = std::max<int64_t>(kmax / 2, 64);
    const SigmaShape cand[4] = {{128, kmax}, {64, kmax}, {128, khalf}, {64, khalf}};
    // every 8th output (16th for lists of over a million products)
    const int stride = tl.outs.size() >= 64 ? (tl.cs.size() > ((size_t)1 << 20) ? 16 : 8) : 1;
    ensure_psi_pieces(P, (int64_t)G * P.dim_pad);
    // a fixed nonzero bf16 pattern in psi's pieces (the sample is timed, not used)
    DMRG_CHECK_CUDA(cudaMemsetAsync(P.ps_hi, 0x3c, (size_t)P.n_ppc * 2, P.stream));
    DMRG_CHECK_CUDA(cudaMemsetAsync(P.ps_lo, 0x3c, (size_t)P.n_ppc * 2 * P.lo_pieces(), P.stream));
    double* out = P.alloc(std::max<int64_t>(P.dim, 1));
    cudaEvent_t e0 = P.take_event(), e1 = P.take_event();
    double best = 0.0;
    int bi = 0;
    ProductList smp;
    try {
        for (int c = 0; c < 4; ++c) {
            smp.clear();
            smp.outs = tl.outs;
            for (const Contrib& x : tl.cs)
                if (x.out % stride == 0) smp.cs.push_back(x);
            smp.lower_tma(BUF_SCR, BUF_ID, P.id_n, cap, cand[c].kchunk, TC_ATOMIC_F64, vs, G, cand[c].tn);
            smp.cs.clear();
            ensure_scratch(P, (int64_t)G * smp.scratch_elems);
            for (auto& ch : smp.tchunks) {
                ch.first.upload(P.stream);
                ch.second.upload(P.stream);
            }
            const TcBufs tb = sigma_bufs(P, k, out);
            smp.maps.encode_upload(tb, P.nsplit, P.stream);
            tc_prepare(P.nsplit);
            float msb = 0.f;
            for (int rep = 0; rep < 2; ++rep) {  // a warm-up run, then the timed one
                DMRG_CHECK_CUDA(cudaEventRecord(e0, P.stream));
                smp.run_tma(tb, 1, P.nsplit, P.stream);
                DMRG_CHECK_CUDA(cudaEventRecord(e1, P.stream));
                DMRG_CHECK_CUDA(cudaEventSynchronize(e1));
                DMRG_CHECK_CUDA(cudaEventElapsedTime(&msb, e0, e1));
            }
            P.check_device_error();
            P.stats.tune_cand_ms[c] = msb;
            if (c == 0 || msb < 0.98 * best) {
                best = msb;
                bi = c;
            }
        }
    } catch (...) {
        smp.clear();
        P.free(out, std::max<int64_t>(P.dim, 1));
        P.ev_pool.push_back(e0);
        P.ev_pool.push_back(e1);
        throw;
    }
    smp.clear();
    P.free(out, std::max<int64_t>(P.dim, 1));
    P.ev_pool.push_back(e0);
    P.ev_pool.push_back(e1);
    P.tune_cache[key] = {cand[bi].tn, cand[bi].kchunk};
    ++P.stats.tunes;
    P.stats.ms_tune += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return cand[bi];
}

}  // namespace

void free_block(Plan& P, std::unique_ptr<Block>& b) {
    if (!b) return;
    tier_release(P, *b);
    P.free(b->d, b->n);
    P.free_bf16(b->h, b->n);
    P.free_lo(b->l, b->n);
    b.reset();
}

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

void ensure_ident(Plan& P, int n) {
    n = (int)round_up(std::max(n, 64), 8);
    if (n > P.ident_n) {
        P.free(P.d_ident, (int64_t)P.ident_n * P.ident_n);
        P.ident_n = n;
        P.d_ident = P.alloc((int64_t)n * n);
        dev_identity(P.d_ident, n, P.stream);
    }
    if (P.mixed() && P.id_n != P.ident_n) {
        P.free_bf16(P.id_hi, (int64_t)P.id_n * P.id_n);
        P.free_lo(P.id_lo, (int64_t)P.id_n * P.id_n);
        P.id_n = P.ident_n;
        const int64_t nn = (int64_t)P.id_n * P.id_n;
        P.id_hi = P.alloc_bf16(nn);
        P.id_lo = P.alloc_lo(nn);
        dev_split_f64(P.d_ident, 1, (int)nn, nn, P.id_hi, P.id_lo, nn, P.stream, P.lo2(P.id_lo, nn));
    }
}

void ensure_scratch(Plan& P, int64_t n) {
    if (P.mixed()) {
        if (n <= P.n_spc) return;
        P.free_bf16(P.s_hi, P.n_spc);
        P.free_lo(P.s_lo, P.n_spc);
        P.n_spc = n;
        P.s_hi = P.alloc_bf16(n);
        P.s_lo = P.alloc_lo(n);
        return;
    }
    if (n <= P.n_scratch) return;
    P.free(P.d_scratch, P.n_scratch);
    P.n_scratch = n;
    P.d_scratch = P.alloc(n);
}

void ensure_scratch_f64(Plan& P, int64_t n) {
    if (n <= P.n_scratch) return;
    P.free(P.d_scratch, P.n_scratch);
    P.n_scratch = n;
    P.d_scratch = P.alloc(n);
}

int64_t scratch_cap(const Plan& P) {
    const int64_t esz = P.mixed() ? 4 : 8;  // two bf16 pieces or one double per element
    int64_t cap = P.opt.scratch_bytes > 0 ? P.opt.scratch_bytes / esz : 0;
    if (cap <= 0) cap = std::max<int64_t>((int64_t)1 << 27, P.budget / esz / 12);
    return cap;
}

int64_t scratch_cap_f64(const Plan& P) {
    int64_t cap = P.opt.scratch_bytes > 0 ? P.opt.scratch_bytes / 8 : 0;
    if (cap <= 0) cap = std::max<int64_t>((int64_t)1 << 26, P.budget / 8 / 12);
    return cap;
}

// ---------------------------------------------------------------------------
// Intermediates: Int[rows x nnz] = W[rows x nops] * Family[nops x nnz]
// ---------------------------------------------------------------------------

void interm_bases(Interms& im, const Block* blocks[2]) {
    int64_t total = 0;
    for (auto& IF : im.fams) {
        const Family& f = blocks[IF.owner]->lay.fams[IF.src_fam];
        IF.base = total;
        total += (int64_t)IF.rows.size() * f.stride;
    }
}

void form_interms(Plan& P, Interms& im, const Block* blocks[2], IntermStore& S, double& flops, bool bases_set) {
    if (!bases_set) interm_bases(im, blocks);
    // (im is read-only from here: a host thread may be lowering lists that refer to it)
    int64_t total = 0, wtot = 0;
    for (const auto& IF : im.fams) {
        const Family& f = blocks[IF.owner]->lay.fams[IF.src_fam];
        total += (int64_t)IF.rows.size() * f.stride;
        wtot += (int64_t)IF.rows.size() * round_up(f.nops(), 8);
    }
    free_interms(P, S);
    S.n = std::max<int64_t>(total, 32);
    flops = 0.0;
    if (P.mixed()) {
        S.h = P.alloc_bf16(S.n);
        S.l = P.alloc_lo(S.n);
    }
    if (P.f64_store()) S.d = P.alloc(S.n);
    if (im.fams.empty()) return;
    std::vector<double> W(std::max<int64_t>(wtot, 8), 0.0);
    WorkList wl;
    if (!P.tc_store()) P.f64_tiles(wl);
    int64_t woff = 0;
    for (auto& IF : im.fams) {
        const Family& f = blocks[IF.owner]->lay.fams[IF.src_fam];
        const int nr = (int)IF.rows.size(), no = f.nops();
        const int ldw = P.tc_store() ? (int)round_up(no, 8) : no;
        for (int r = 0; r < nr; ++r)
            for (auto& rc : IF.rows[r]) W[woff + (int64_t)r * ldw + rc.first] += rc.second;
        DMRG_REQUIRE(f.stride < (1LL << 31), DMRG_EINVAL, "operator family too large");
        Seg s{};
        s.a_off = woff;
        s.b_off = f.base;
        s.k = no;
        s.lda = ldw;
        s.ldb = (int)f.stride;
        s.a_buf = BUF_W;
        s.b_buf = (uint8_t)IF.owner;  // BUF_L or BUF_R
        s.alpha = 1.0;
        if (P.tc_store()) wl.add_block(IF.base, BUF_INT, nr, (int)f.nnz, (int)f.stride, {s}, TC_ATOMIC_F64, kChunkTC, 128, 1.0f);
        else wl.add_block(IF.base, BUF_INT, nr, (int)f.nnz, (int)f.stride, {s}, TILE_STORE);
        woff += (int64_t)nr * ldw;
    }
    flops = wl.flops;
    const int64_t wn = (int64_t)W.size();
    if (wn > P.n_wcoef) {
        P.free(P.d_wcoef, P.n_wcoef);
        P.n_wcoef = wn;
        P.d_wcoef = P.alloc(wn);
    }
    DMRG_CHECK_CUDA(cudaMemcpyAsync(P.d_wcoef, W.data(), wn * 8, cudaMemcpyHostToDevice, P.stream));
    wl.upload(P.stream);
    if (P.tc_store()) {
        if (wn > P.n_wpc) {
            P.free_bf16(P.w_hi, P.n_wpc);
            P.free_lo(P.w_lo, P.n_wpc);
            P.n_wpc = wn;
            P.w_hi = P.alloc_bf16(wn);
            P.w_lo = P.alloc_lo(wn);
        }
        dev_split_f64(P.d_wcoef, 1, (int)wn, wn, P.w_hi, P.w_lo, wn, P.stream, P.lo2(P.w_lo, P.n_wpc));
        // FP32 sum of the K-chunks, then split into the bf16 pieces
        double* acc = P.alloc(S.n);  // FP64 sum of the K-chunks, then split into the pieces
        DMRG_CHECK_CUDA(cudaMemsetAsync(acc, 0, S.n * 8, P.stream));
        TcBufs tb = tc_base(P);
        for (int o = 0; o < 2; ++o)
            if (blocks[o]) {
                set_pieces(P, tb, o, blocks[o]->h, blocks[o]->l, blocks[o]->n);
            }
        set_pieces(P, tb, BUF_W, P.w_hi, P.w_lo, P.n_wpc);
        tb.out[BUF_INT] = acc;
        launch_seg_gemm_tc(wl, tb, 1, P.nsplit, P.stream);
        P.check_device_error();
        dev_split_f64_flat(acc, S.n, S.h, S.l, P.stream, P.lo2(S.l, S.n));
        DMRG_CHECK_CUDA(cudaStreamSynchronize(P.stream));
        P.free(acc, S.n);
    } else {
        BufTable bt{};
        bt.p[BUF_L] = blocks[0] ? blocks[0]->d : nullptr;
        bt.p[BUF_R] = blocks[1] ? blocks[1]->d : nullptr;
        bt.p[BUF_INT] = S.d;
        bt.p[BUF_W] = P.d_wcoef;
        launch_seg_gemm_f64(wl, bt, 1, P.stream);
        if (P.mixed()) dev_split_f64_flat(S.d, S.n, S.h, S.l, P.stream, P.lo2(S.l, S.n));
    }
    DMRG_CHECK_CUDA(cudaStreamSynchronize(P.stream));
    wl.release();
}

void free_interms(Plan& P, IntermStore& S) {
    P.free(S.d, S.n);
    P.free_bf16(S.h, S.n);
    P.free_lo(S.l, S.n);
    S.n = 0;
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
    B->n = std::max<int64_t>(B->lay.total, 32);
    if (P.mixed()) {
        B->h = P.alloc_bf16(B->n);
        B->l = P.alloc_lo(B->n);
        DMRG_CHECK_CUDA(cudaMemsetAsync(B->h, 0, B->n * 2, P.stream));
        DMRG_CHECK_CUDA(cudaMemsetAsync(B->l, 0, P.lo_pieces() * B->n * 2, P.stream));
    }
    if (P.f64_store()) {
        B->d = P.alloc(B->n);
        dev_fill(B->d, 0.0, B->n, P.stream);
    }
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

// Device copy of site tensor A[k] with rows padded to 8: key -> (offset, ld).
struct SiteDev {
    double* d = nullptr;
    __nv_bfloat16 *h = nullptr, *l = nullptr;
    int64_t n = 0;
    std::map<std::array<int, 3>, std::pair<int64_t, int>> off;
};

static SiteDev upload_site(Plan& P, int k) {
    SiteDev S;
    int64_t tot = 0;
    const auto& bl = P.mps.bonds[k - 1];
    const auto& br = P.mps.bonds[k];
    for (auto& kv : P.mps.sites[k]) {
        const int dl = bl[kv.first[0]][2], dr = br[kv.first[2]][2];
        const int ld = (int)round_up(dr, 8);
        S.off[kv.first] = {tot, ld};
        tot += (int64_t)dl * ld;
    }
    S.n = std::max<int64_t>(tot, 8);
    std::vector<double> host(S.n, 0.0);
    for (auto& kv : P.mps.sites[k]) {
        const int dl = bl[kv.first[0]][2], dr = br[kv.first[2]][2];
        const auto o = S.off[kv.first];
        for (int a = 0; a < dl; ++a)
            std::copy(kv.second.begin() + (int64_t)a * dr, kv.second.begin() + (int64_t)(a + 1) * dr,
                      host.begin() + o.first + (int64_t)a * o.second);
    }
    S.d = P.alloc(S.n);
    DMRG_CHECK_CUDA(cudaMemcpyAsync(S.d, host.data(), S.n * 8, cudaMemcpyHostToDevice, P.stream));
    if (P.mixed()) {
        S.h = P.alloc_bf16(S.n);
        S.l = P.alloc_lo(S.n);
        dev_split_f64(S.d, 1, (int)S.n, S.n, S.h, S.l, S.n, P.stream, P.lo2(S.l, S.n));
    }
    DMRG_CHECK_CUDA(cudaStreamSynchronize(P.stream));
    return S;
}

static void free_site(Plan& P, SiteDev& S) {
    P.free(S.d, S.n);
    P.free_bf16(S.h, S.n);
    P.free_lo(S.l, S.n);
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
    IntermStore IS;
    double fl_int = 0.0;
    form_interms(P, rp.interms, blocks, IS, fl_int);
    SiteDev A = upload_site(P, m);
    out->n = std::max<int64_t>(OL.total, 32);

    const auto host0 = std::chrono::steady_clock::now();
    double host_lower_ms = 0.0;
    ProductList pl;
    std::vector<std::array<int, 3>> keys;
    for (auto& kv : P.mps.sites[m]) keys.push_back(kv.first);
    const auto& bl = P.mps.bonds[m - 1];
    const auto& br = P.mps.bonds[m];
    const int nl = (int)bl.size(), nrb = (int)br.size();
    // dense tables: site block (il, n, ir) -> (offset, ld); bra lookups
    // forward (jl, c') -> jr and backward (n', jr) -> jl
    std::vector<std::pair<int64_t, int>> site_at((size_t)nl * 4 * nrb, {-1, 0});
    std::vector<int> fwd_bra((size_t)nl * 4, -1), bwd_bra((size_t)4 * nrb, -1);
    for (auto& kk : keys) {
        site_at[((size_t)kk[0] * 4 + kk[1]) * nrb + kk[2]] = A.off[kk];
        fwd_bra[(size_t)kk[0] * 4 + kk[1]] = kk[2];
        bwd_bra[(size_t)kk[1] * nrb + kk[2]] = kk[0];
    }
    auto site_view = [&](int il, int n, int ir, bool tr) {
        View v;
        const auto& at = site_at[((size_t)il * 4 + n) * nrb + ir];
        v.buf = BUF_PSI;
        v.off = at.first;
        v.ld = at.second;
        v.tr = tr;
        return v;
    };
    const int nxb = XL.basis.size();
    std::vector<OpLookup> xcache(nxb);
    std::vector<int> out_of_pair;
    for (int t = 0; t < (int)rp.targets.size(); ++t) {
        const RenormTarget& T = rp.targets[t];
        auto fr = OL.find(T.key);
        const Family& of = OL.fams[fr.first];
        const int64_t obase = of.base + (int64_t)fr.second * of.stride;
        out_of_pair.assign(of.bra.size(), -1);  // pair of the target -> output block
        for (const Term2& term : T.terms) {
            const LocalOp& M = rp.site.ops[term.site];
            const int parX = ref_parity(XL, rp.interms, term.X);
            for (int i = 0; i < nxb; ++i) xcache[i] = lookup(XL, rp.interms, term.X, i, BUF_L);
            for (auto& kk : keys) {
                const int il = kk[0], n = kk[1], ir = kk[2];
                if (forward) {
                    // ket component (il, n) of X.C -> new sector ir; X acts on il
                    const OpLookup& ox = xcache[il];
                    if (!ox.ok) continue;
                    const int jl = ox.j;
                    for (int c2 = 0; c2 < 4; ++c2) {
                        const double mv = M.at(c2, n);
                        if (mv == 0.0) continue;
                        const int jr = fwd_bra[(size_t)jl * 4 + c2];
                        if (jr < 0) continue;
                        const int pr = of.pair_of_ket[ir];
                        if (pr < 0 || of.bra[pr] != jr) continue;
                        const int dl = bl[il][2], djl = bl[jl][2], dr = br[ir][2], djr = br[jr][2];
                        const double zeta = (M.parity && (XL.basis.qn[il].n & 1)) ? -1.0 : 1.0;
                        int o = out_of_pair[pr];
                        if (o < 0) {
                            o = (int)pl.outs.size();
                            out_of_pair[pr] = o;
                            pl.outs.push_back({BUF_R, obase + of.off[pr], djr, dr, of.ld[pr]});
                        }
                        Contrib c;
                        c.out = o;
                        c.P = site_view(jl, c2, jr, true);  // A(jl,c2,jr)^T : djr x djl
                        c.Q = ox.v;                          // X_eff : djl x dl
                        c.R = site_view(il, n, ir, false);   // A(il,n,ir) : dl x dr
                        c.m = djr;
                        c.k1 = djl;
                        c.k2 = dl;
                        c.n = dr;
                        c.alpha = term.c * zeta * mv;
                        pl.cs.push_back(c);
                    }
                } else {
                    // ket component (n, ir) of C.X -> new sector il; X acts on ir
                    const OpLookup& ox = xcache[ir];
                    if (!ox.ok) continue;
                    const int jr = ox.j;
                    for (int n2 = 0; n2 < 4; ++n2) {
                        const double mv = M.at(n2, n);
                        if (mv == 0.0) continue;
                        const int jl = bwd_bra[(size_t)n2 * nrb + jr];
                        if (jl < 0) continue;
                        const int pr = of.pair_of_ket[il];
                        if (pr < 0 || of.bra[pr] != jl) continue;
                        const int dl = bl[il][2], djl = bl[jl][2], dr = br[ir][2], djr = br[jr][2];
                        const double zeta = (parX && (kSiteQN[n].n & 1)) ? -1.0 : 1.0;
                        int o = out_of_pair[pr];
                        if (o < 0) {
                            o = (int)pl.outs.size();
                            out_of_pair[pr] = o;
                            pl.outs.push_back({BUF_R, obase + of.off[pr], djl, dl, of.ld[pr]});
                        }
                        Contrib c;
                        c.out = o;
                        c.P = site_view(jl, n2, jr, false);  // A(jl,n2,jr) : djl x djr
                        c.Q = ox.v;                           // X_eff : djr x dr
                        c.R = site_view(il, n, ir, true);     // A(il,n,ir)^T : dr x dl
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
    const int64_t cap = P.tc_store() ? scratch_cap(P) : scratch_cap_f64(P);
    if (P.tc_store()) {
        // the cp.async-staged engine: renormalisation lists hold many short
        // products (K-chunks of 256), where it measured faster than the
        // TMA-staged engine of sigma (map encoding and lowering cost included)
        pl.lower_tc(BUF_SCR, BUF_ID, P.id_n, cap, kChunkTC, TC_ATOMIC_F64);
        host_lower_ms = host_ms_since(host0);
        P.stats.ms_host_plan += host_lower_ms;
        ensure_scratch(P, std::max<int64_t>(pl.scratch_elems, 8));
        pl.upload(P.stream);
        double* acc = P.alloc(out->n);
        DMRG_CHECK_CUDA(cudaMemsetAsync(acc, 0, out->n * 8, P.stream));
        TcBufs tb = tc_base(P);
        set_pieces(P, tb, BUF_L, X.h, X.l, X.n);
        set_pieces(P, tb, BUF_INT, IS.h, IS.l, IS.n);
        set_pieces(P, tb, BUF_PSI, A.h, A.l, A.n);
        set_pieces(P, tb, BUF_SCR, P.s_hi, P.s_lo, P.n_spc);
        set_pieces(P, tb, BUF_ID, P.id_hi, P.id_lo, (int64_t)P.id_n * P.id_n);
        tb.out[BUF_R] = acc;
        set_out_pieces(P, tb, BUF_SCR, P.s_hi, P.s_lo, P.n_spc);
        pl.run_tc(tb, 1, P.nsplit, P.stream);
        P.check_device_error();
        out->h = P.alloc_bf16(out->n);
        out->l = P.alloc_lo(out->n);
        dev_split_f64_flat(acc, out->n, out->h, out->l, P.stream, P.lo2(out->l, out->n));
        DMRG_CHECK_CUDA(cudaStreamSynchronize(P.stream));
        P.free(acc, out->n);
    } else {
        P.f64_tiles(pl);
        pl.lower(BUF_SCR, BUF_ID, P.ident_n, cap, kChunkF64);
        host_lower_ms = host_ms_since(host0);
        P.stats.ms_host_plan += host_lower_ms;
        ensure_scratch_f64(P, std::max<int64_t>(pl.scratch_elems, 1));
        pl.upload(P.stream);
        out->d = P.alloc(out->n);
        DMRG_CHECK_CUDA(cudaMemsetAsync(out->d, 0, out->n * 8, P.stream));
        BufTable bt{};
        bt.p[BUF_L] = X.d;
        bt.p[BUF_R] = out->d;
        bt.p[BUF_INT] = IS.d;
        bt.p[BUF_PSI] = A.d;
        bt.p[BUF_SCR] = P.d_scratch;
        bt.p[BUF_ID] = P.d_ident;
        pl.run(bt, 1, P.stream);
        if (P.mixed()) {  // bf16 pieces of the FP64 store for the tensor-core sigma
            out->h = P.alloc_bf16(out->n);
            out->l = P.alloc_lo(out->n);
            dev_split_f64_flat(out->d, out->n, out->h, out->l, P.stream, P.lo2(out->l, out->n));
        }
    }
    cudaEventRecord(e1, P.stream);
    DMRG_CHECK_CUDA(cudaStreamSynchronize(P.stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    P.stats.ms_renorm += ms;
    P.stats.renorm_flops_last = pl.flops + fl_int;
    P.stats.renorm_flops_total += pl.flops + fl_int;
    if (P.opt.verbose)
        fprintf(stderr, "[dmrg] renormalise site %d (%s): %.0f ms, of which host lowering %.0f ms; %zu products, "
                        "%.3g FLOP\n",
                m, forward ? "forward" : "backward", ms, host_lower_ms, pl.cs.size(), pl.flops + fl_int);
    pl.release();
    free_interms(P, IS);
    free_site(P, A);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return out;
}

// ---------------------------------------------------------------------------
// Current bond
// ---------------------------------------------------------------------------

void ensure_env(Plan& P, int k) {
    const int K = P.K;
    if (!P.left[0]) P.left[0] = make_vacuum(P, false);
    const int m = k - 1;
    int have = m;
    while (have > 0 && !P.left[have]) --have;
    // keep the block next to the new one (a step back needs it) and free the
    // rest; sweeps keep them all, with the host tier off the device
    const bool tier = P.opt.keep_envs && P.opt.host_tier;
    for (int j = have + 1; j <= m; ++j) {
        tier_need(P, *P.left[j - 1]);
        P.left[j] = renormalise(P, *P.left[j - 1], j, true);
        if (!P.opt.keep_envs && j - 1 >= 1 && j - 1 < m - 1) free_block(P, P.left[j - 1]);
        if (tier && j - 1 < m - 1) {
            tier_out(P, *P.left[j - 1]);
            tier_drain(P, false);
        }
    }
    if (!P.right[K]) P.right[K] = make_vacuum(P, true);
    const int mr = k + 1;
    int haver = mr;
    while (haver < K && !P.right[haver]) ++haver;
    for (int j = haver - 1; j >= mr; --j) {
        tier_need(P, *P.right[j + 1]);
        P.right[j] = renormalise(P, *P.right[j + 1], j + 1, false);
        if (!P.opt.keep_envs && j + 1 <= K - 1 && j + 1 > mr + 1) free_block(P, P.right[j + 1]);
        if (tier && j + 1 > mr + 1) {
            tier_out(P, *P.right[j + 1]);
            tier_drain(P, false);
        }
    }
    tier_need(P, *P.left[m]);
    tier_need(P, *P.right[mr]);
}

void build_layout(Plan& P, int k) {
    P.layout.clear();
    P.sector_of.clear();
    P.sector_idx.assign(16 * std::max<size_t>(P.mps.bonds[k - 1].size(), 1), -1);
    const auto& bl = P.mps.bonds[k - 1];
    const auto& br = P.mps.bonds[k + 1];
    std::map<std::pair<int, int>, int> ridx;
    for (int i = 0; i < (int)br.size(); ++i) ridx[{br[i][0], br[i][1]}] = i;
    int64_t off = 0, poff = 0;
    for (int il = 0; il < (int)bl.size(); ++il)
        for (int y = 0; y < 16; ++y) {
            QN q = QN(bl[il][0], bl[il][1]) + kSiteQN[y / 4] + kSiteQN[y % 4];
            auto it = ridx.find({q.n, q.s});
            if (it == ridx.end()) continue;
            Plan::Sector s{il, y, it->second, off, bl[il][2], br[it->second][2], poff};
            P.sector_of[{il, y}] = (int)P.layout.size();
            P.sector_idx[16 * il + y] = (int)P.layout.size();
            P.layout.push_back(s);
            off += (int64_t)s.dl * s.dr;
            poff += (int64_t)s.dl * round_up(s.dr, 8);
        }
    P.dim = off;
    P.dim_pad = std::max<int64_t>(poff, 8);
}

void set_bond(Plan& P, int k) {
    DMRG_REQUIRE(k >= 1 && k <= P.K - 1, DMRG_EINVAL, "bond index out of range");
    DMRG_REQUIRE(k == P.mps.center, DMRG_EINVAL,
                 "bond " + std::to_string(k) + " is not the MPS centre " + std::to_string(P.mps.center));
    if (P.opt.host_tier) tier_drain(P, true);  // evictions started at the previous bond
    ensure_env(P, k);
    const Block& L = *P.left[k - 1];
    const Block& R = *P.right[k + 1];
    build_layout(P, k);
    build_sigma_terms(P.I, L.lay, R.lay, k, P.sp);
    const Block* blocks[2] = {&L, &R};
    interm_bases(P.sp.interms, blocks);  // offsets the sigma lists refer to
    int maxd = std::max({L.lay.basis.dmax(), R.lay.basis.dmax(), 1});
    ensure_ident(P, maxd);
    P.sigma_fp64_ready = false;
    P.sigma_units_pl.clear();
    P.sigma_units_ready = false;

    // sigma contributions (FP64 views; the bf16 copy of psi is padded)
    ProductList& pl = P.sigma_pl;
    ProductList& tl = P.sigma_tc;
    const LocalOps& Y = P.sp.y;
    // the blocks of a term's operators depend only on the ket sector of their
    // side; terms are taken in blocks on host threads and their contributions
    // concatenated in term order
    const int nbl = L.lay.basis.size(), nbr = R.lay.basis.size();
    const size_t nterm = P.sp.terms.size();
    const size_t tblk = std::max<size_t>(1, (nterm + 63) / 64);
    const size_t nblk = (nterm + tblk - 1) / tblk;
    // vectors per launch (block Davidson passes up to n_roots at once)
    const int G = std::max(1, P.opt.n_roots);
    int64_t vs[kMaxBufs] = {};
    vs[BUF_PSI] = P.dim_pad;
    const int64_t cap = std::max<int64_t>(scratch_cap(P) / G, 1 << 20);
    SigmaShape shape{128, P.opt.tc_kchunk > 0 ? P.opt.tc_kchunk : (P.nsplit == 3 ? kChunkSigmaX6 : kChunkSigmaTC)};
    if (P.opt.sigma_tile_n > 0) shape.tn = P.opt.sigma_tile_n;
    int64_t nitems = 0;
    bool tune_later = false;
    double t_terms = 0.0, t_lower = 0.0, t_count = 0.0, plan_ms = 0.0;
    auto lower_and_count = [&]() {
        const auto c0 = std::chrono::steady_clock::now();
        tl.chunk_per_term = P.opt.sigma_per_term != 0;
        tl.lower_tma(BUF_SCR, BUF_ID, P.id_n, cap, shape.kchunk, TC_ATOMIC_F64, vs, G, shape.tn);
        t_lower += host_ms_since(c0);
        const auto c1 = std::chrono::steady_clock::now();
        P.stats.sigma_tile_n = shape.tn;
        P.stats.sigma_kchunk = shape.kchunk;
        tl.cs.clear();
        for (int ph = 0; ph < 2; ++ph) {
            P.stats.sigma_tiles[ph] = P.stats.sigma_stages[ph] = 0;
            P.stats.sigma_load_bytes[ph][0] = P.stats.sigma_load_bytes[ph][1] = 0.0;
        }
        P.stats.sigma_mma_flops = 0.0;
        // per (chunk, phase) on host threads, summed in order afterwards
        struct TileCount {
            int64_t tiles = 0, stages = 0;
            double mma = 0.0, load[2] = {0.0, 0.0};
        };
        std::vector<TileCount> cnt(2 * tl.tchunks.size());
        parallel_for(cnt.size(), [&](size_t x) {
            const int ph = (int)(x & 1);
            const TmaWorkList& w = ph ? tl.tchunks[x / 2].second : tl.tchunks[x / 2].first;
            TileCount& c = cnt[x];
            c.tiles = (int64_t)w.tiles.size();
            for (const Tile& t : w.tiles) {
                int64_t kk = 0;
                for (int q = t.seg_beg; q < t.seg_end; ++q) kk += round_up(w.segs[q].k, 16);
                for (int q = t.seg_beg; q < t.seg_end; ++q) c.stages += (w.segs[q].k + 63) / 64;
                c.mma += 2.0 * 128 * 128 * (double)kk;
                // operand bytes the TMA loads for this tile (boxes of 128-byte
                // rows, one per piece), split into scratch and everything else
                const int nA = (t.m - t.m0 > 64) ? 2 : 1, nB = (std::min(t.tn, t.n - t.n0) > 64) ? 2 : 1;
                for (int q = t.seg_beg; q < t.seg_end; ++q) {
                    const TSeg& g = w.segs[q];
                    const double st = (double)((g.k + 63) / 64) * P.nsplit * 128.0;
                    c.load[tl.maps.keys[g.a_map].buf == BUF_SCR ? 1 : 0] += st * nA * g.a_br;
                    c.load[tl.maps.keys[g.b_map].buf == BUF_SCR ? 1 : 0] += st * nB * g.b_br;
                }
            }
        });
        for (size_t x = 0; x < cnt.size(); ++x) {
            const int ph = (int)(x & 1);
            P.stats.sigma_tiles[ph] += cnt[x].tiles;
            P.stats.sigma_stages[ph] += cnt[x].stages;
            P.stats.sigma_mma_flops += cnt[x].mma;
            P.stats.sigma_load_bytes[ph][0] += cnt[x].load[0];
            P.stats.sigma_load_bytes[ph][1] += cnt[x].load[1];
        }
        t_count = host_ms_since(c1);
    };
    // The host part of the sigma plan (contributions, their lowering into
    // tiles and tensor maps, counts) reads host structures only and runs on a
    // thread while the GPU forms the intermediates; the tuner, allocations and
    // uploads follow on this thread.
    auto host_plan = [&]() {
        const auto h0 = std::chrono::steady_clock::now();
        pl.clear();
        for (const Plan::Sector& s : P.layout) pl.outs.push_back({BUF_OUT, s.off, s.dl, s.dr, s.dr});
        std::vector<std::vector<Contrib>> part(nblk);
        parallel_for(nblk, [&](size_t b) {
            std::vector<OpLookup> lcache(nbl), rcache(nbr);
            std::vector<Contrib>& out = part[b];
            for (size_t ti = b * tblk; ti < std::min(nterm, (b + 1) * tblk); ++ti) {
                const Term3& t = P.sp.terms[ti];
                const LocalOp& M = Y.ops[t.y];
                const int pR = ref_parity(R.lay, P.sp.interms, t.R);
                for (int i = 0; i < nbl; ++i) lcache[i] = lookup(L.lay, P.sp.interms, t.L, i, BUF_L);
                for (int i = 0; i < nbr; ++i) rcache[i] = lookup(R.lay, P.sp.interms, t.R, i, BUF_R);
                for (size_t si = 0; si < P.layout.size(); ++si) {
                    const Plan::Sector& s = P.layout[si];
                    const OpLookup& ol = lcache[s.il];
                    if (!ol.ok) continue;
                    const OpLookup& orr = rcache[s.ir];
                    if (!orr.ok) continue;
                    const int nl = L.lay.basis.qn[s.il].n;
                    const int ny = kSiteQN[s.y / 4].n + kSiteQN[s.y % 4].n;
                    for (int y2 = 0; y2 < 16; ++y2) {
                        const double mv = M.at(y2, s.y);
                        if (mv == 0.0) continue;
                        const int os = P.sector_idx[16 * ol.j + y2];
                        if (os < 0) continue;
                        const Plan::Sector& o = P.layout[os];
                        DMRG_REQUIRE(o.ir == orr.j, DMRG_EINVAL, "sigma term breaks the symmetry");
                        const int e = M.parity * nl + pR * (nl + ny);
                        const double zeta = (e & 1) ? -1.0 : 1.0;
                        Contrib c;
                        c.out = os;
                        c.P = ol.v;  // O^L_eff : d_jl x d_il
                        c.Q.buf = BUF_PSI;
                        c.Q.off = s.off;
                        c.Q.ld = s.dr;  // Psi_s : d_il x d_ir
                        c.R = orr.v.T();  // (O^R_eff)^T : d_ir x d_jr
                        c.m = o.dl;
                        c.k1 = s.dl;
                        c.k2 = s.dr;
                        c.n = o.dr;
                        c.alpha = t.c * zeta * mv;
                        c.qsec = (int)si;
                        c.term = (int)ti;
                        out.push_back(c);
                    }
                }
            }
        });
        size_t ntot = 0;
        for (auto& v : part) ntot += v.size();
        pl.cs.reserve(ntot);
        for (auto& v : part) pl.cs.insert(pl.cs.end(), v.begin(), v.end());
        nitems = (int64_t)ntot;
        if (P.mixed()) {
            tl.clear();
            tl.outs = pl.outs;
            // the tensor-core list reads psi from its padded bf16 copy
            tl.cs.resize(pl.cs.size());
            const size_t cb = 1 << 16;
            parallel_for((pl.cs.size() + cb - 1) / cb, [&](size_t b) {
                for (size_t x = b * cb; x < std::min(pl.cs.size(), (b + 1) * cb); ++x) {
                    Contrib c = pl.cs[x];
                    const Plan::Sector& s = P.layout[c.qsec];
                    c.Q.off = s.poff;
                    c.Q.ld = (int)round_up(s.dr, 8);
                    tl.cs[x] = c;
                }
            });
            t_terms = host_ms_since(h0);
            // lists of over a million products keep the default shape: it won every
            // measurement at that size (K = 54 and K = 73 middle bonds), and the
            // timing of the candidates costs 0.3-1 s per new bond there
            tune_later = P.opt.sigma_tile_n <= 0 && P.opt.sigma_tune && P.opt.tc_kchunk <= 0 &&
                         !P.opt.sigma_per_term && tl.cs.size() <= ((size_t)1 << 20);
            if (!tune_later) lower_and_count();
        } else {
            t_terms = host_ms_since(h0);
            P.f64_tiles(pl);
            pl.lower(BUF_SCR, BUF_ID, P.ident_n, scratch_cap(P), kChunkF64);
        }
        plan_ms = host_ms_since(h0);
    };
    std::exception_ptr plan_err;
    int device = 0;  // the thread frees the old lists' device arrays on the plan's device
    DMRG_CHECK_CUDA(cudaGetDevice(&device));
    std::thread planner([&]() {
        try {
            DMRG_CHECK_CUDA(cudaSetDevice(device));
            host_plan();
        } catch (...) {
            plan_err = std::current_exception();
        }
    });
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, P.stream);
    double fl = 0.0;
    try {
        form_interms(P, P.sp.interms, blocks, P.interm, fl, true);
        cudaEventRecord(e1, P.stream);
        DMRG_CHECK_CUDA(cudaStreamSynchronize(P.stream));
    } catch (...) {
        planner.join();
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    planner.join();
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (plan_err) std::rethrow_exception(plan_err);
    P.stats.ms_interm += ms;
    P.stats.interm_flops = fl;
    P.stats.interm_flops_total += fl;
    const int esz = (P.mixed() ? 2 * (1 + P.lo_pieces()) : 0) + (P.f64_store() ? 8 : 0);
    P.stats.interm_bytes = P.interm.n * esz;
    P.stats.store_bytes = (L.n + R.n) * esz;
    const auto hs0 = std::chrono::steady_clock::now();
    if (P.mixed()) {
        double t_tune = 0.0;
        if (tune_later) {
            const auto c0 = std::chrono::steady_clock::now();
            shape = tune_sigma_shape(P, k, tl, cap, shape.kchunk, vs, G);
            t_tune = host_ms_since(c0);
            lower_and_count();
        }
        const auto u0 = std::chrono::steady_clock::now();
        ensure_scratch(P, (int64_t)G * tl.scratch_elems);
        ensure_psi_pieces(P, (int64_t)G * P.dim_pad);
        for (auto& ch : tl.tchunks) {
            ch.first.upload(P.stream);
            ch.second.upload(P.stream);
        }
        tl.maps.encode_upload(sigma_bufs(P, k, nullptr), P.nsplit, P.stream);
        if (P.opt.verbose)
            fprintf(stderr, "[dmrg] bond %d sigma planning: terms %.0f ms, tuning %.0f ms, lowering %.0f ms, "
                            "counts %.0f ms, upload %.0f ms (%zu chunks)\n",
                    k, t_terms, t_tune, t_lower, t_count, host_ms_since(u0), tl.tchunks.size());
        P.stats.sigma_maps = (int64_t)tl.maps.keys.size();
        P.stats.sigma_flops = tl.flops;
        // padded bf16 copy of psi: one split job per sector
        std::vector<SplitJob> jobs;
        for (const Plan::Sector& s : P.layout)
            jobs.push_back({s.off, s.poff, s.dl, s.dr, s.dr, (int)round_up(s.dr, 8)});
        if (P.d_psi_jobs) cudaFree(P.d_psi_jobs);
        P.n_psi_jobs = (int)jobs.size();
        DMRG_CHECK_CUDA(cudaMalloc(&P.d_psi_jobs, std::max<size_t>(jobs.size(), 1) * sizeof(SplitJob)));
        if (!jobs.empty())
            DMRG_CHECK_CUDA(cudaMemcpyAsync(P.d_psi_jobs, jobs.data(), jobs.size() * sizeof(SplitJob),
                                            cudaMemcpyHostToDevice, P.stream));
    } else {
        ensure_scratch(P, std::max<int64_t>(pl.scratch_elems, 1));
        pl.upload(P.stream);
        P.sigma_fp64_ready = true;
        P.stats.sigma_flops = pl.flops;
    }
    P.stats.n_terms = (int64_t)P.sp.terms.size();
    P.stats.n_items = nitems;
    P.stats.sigma_chunks = (int)(P.mixed() ? P.sigma_tc.tchunks.size() : P.sigma_pl.chunks.size());

    // diag(H_eff): terms whose three factors all conserve the quantum numbers
    ProductList& hl = P.hdiag_pl;
    hl.clear();
    {
        WorkList w;
        std::vector<std::vector<Seg>> per(P.layout.size());
        // terms in blocks on host threads; each block's (sector, segment) pairs
        // are appended in term order
        std::vector<std::vector<std::pair<int, Seg>>> dpart(nblk);
        parallel_for(nblk, [&](size_t blk) {
            std::vector<OpLookup> lcache(nbl), rcache(nbr);
            for (size_t ti = blk * tblk; ti < std::min(nterm, (blk + 1) * tblk); ++ti) {
                const Term3& t = P.sp.terms[ti];
                const LocalOp& M = Y.ops[t.y];
                if (M.dq != QN(0, 0)) continue;
                const int pR = ref_parity(R.lay, P.sp.interms, t.R);
                for (int i = 0; i < nbl; ++i) lcache[i] = lookup(L.lay, P.sp.interms, t.L, i, BUF_L);
                for (int i = 0; i < nbr; ++i) rcache[i] = lookup(R.lay, P.sp.interms, t.R, i, BUF_R);
                for (size_t si = 0; si < P.layout.size(); ++si) {
                    const Plan::Sector& s = P.layout[si];
                    const double mv = M.at(s.y, s.y);
                    if (mv == 0.0) continue;
                    const OpLookup& ol = lcache[s.il];
                    if (!ol.ok || ol.j != s.il) continue;
                    const OpLookup& orr = rcache[s.ir];
                    if (!orr.ok || orr.j != s.ir) continue;
                    const int nl = L.lay.basis.qn[s.il].n;
                    const int ny = kSiteQN[s.y / 4].n + kSiteQN[s.y % 4].n;
                    const int e = M.parity * nl + pR * (nl + ny);
                    const double zeta = (e & 1) ? -1.0 : 1.0;
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
                    dpart[blk].push_back({(int)si, sg});
                }
            }
        });
        for (auto& v : dpart)
            for (auto& x : v) per[x.first].push_back(x.second);
        w.rank1 = true;  // every segment is one diagonal outer product (k = 1)
        for (size_t si = 0; si < P.layout.size(); ++si) {
            const Plan::Sector& s = P.layout[si];
            w.add_block(s.off, BUF_OUT, s.dl, s.dr, s.dr, per[si], TILE_STORE);
        }
        hl.chunks.emplace_back(WorkList(), std::move(w));
        hl.upload(P.stream);
    }
    // per-sector quantum numbers of the left block (features of the learned preconditioner)
    {
        std::vector<int64_t> off(P.layout.size() + 1, 0);
        std::vector<float> q(2 * std::max<size_t>(P.layout.size(), 1), 0.f);
        const auto& bl = P.mps.bonds[k - 1];
        for (size_t i = 0; i < P.layout.size(); ++i) {
            off[i] = P.layout[i].off;
            q[2 * i] = (float)bl[P.layout[i].il][0] / (float)std::max(P.N, 1);
            q[2 * i + 1] = (float)bl[P.layout[i].il][1] / (float)std::max(P.N, 1);
        }
        off[P.layout.size()] = P.dim;
        Mlp& m = P.mlp;
        cudaFree(m.d_sec_off);
        cudaFree(m.d_sec_q);
        m.n_sec = (int)std::max<size_t>(P.layout.size(), 1);
        DMRG_CHECK_CUDA(cudaMalloc(&m.d_sec_off, off.size() * sizeof(int64_t)));
        DMRG_CHECK_CUDA(cudaMalloc(&m.d_sec_q, q.size() * sizeof(float)));
        DMRG_CHECK_CUDA(cudaMemcpyAsync(m.d_sec_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                                        P.stream));
        DMRG_CHECK_CUDA(
            cudaMemcpyAsync(m.d_sec_q, q.data(), q.size() * sizeof(float), cudaMemcpyHostToDevice, P.stream));
    }
    P.stats.ms_host_plan += plan_ms + host_ms_since(hs0);
    P.drop_graphs();  // captured for the previous bond's work lists
    P.bond = k;
    DMRG_CHECK_CUDA(cudaStreamSynchronize(P.stream));
}

// FP64 engine tables (the operator buffers are bf16 pieces in mixed mode)
BufTable bond_buffers(Plan& P, const double* psi, double* out) {
    BufTable bt{};
    const Block& L = *P.left[P.bond - 1];
    const Block& R = *P.right[P.bond + 1];
    if (P.tc_store()) {
        bt.p[BUF_L] = (double*)L.h;
        bt.lo[BUF_L] = L.l;
        bt.p[BUF_R] = (double*)R.h;
        bt.lo[BUF_R] = R.l;
        bt.p[BUF_INT] = (double*)P.interm.h;
        bt.lo[BUF_INT] = P.interm.l;
        if (P.nsplit == 3) {
            bt.pstride[BUF_L] = L.n;
            bt.pstride[BUF_R] = R.n;
            bt.pstride[BUF_INT] = P.interm.n;
        }
        bt.pmask = (1u << BUF_L) | (1u << BUF_R) | (1u << BUF_INT);
    } else {
        bt.p[BUF_L] = L.d;
        bt.p[BUF_R] = R.d;
        bt.p[BUF_INT] = P.interm.d;
    }
    bt.p[BUF_PSI] = const_cast<double*>(psi);
    bt.p[BUF_SCR] = P.d_scratch;
    bt.p[BUF_ID] = P.d_ident;
    bt.p[BUF_OUT] = out;
    bt.vstride[BUF_PSI] = P.dim;
    bt.vstride[BUF_OUT] = P.dim;
    bt.vstride[BUF_SCR] = P.sigma_pl.scratch_elems;
    return bt;
}

// sigma in FP64 arithmetic over the stored operators (exact upcast of the
// bf16 pieces in mixed mode)
void sigma_fp64(Plan& P, const double* psi, double* out, int nvec, cudaStream_t st) {
    DMRG_REQUIRE(P.bond > 0, DMRG_EINVAL, "no current bond (call dmrg_set_bond)");
    if (!P.sigma_fp64_ready) {
        P.f64_tiles(P.sigma_pl);
        P.sigma_pl.lower(BUF_SCR, BUF_ID, P.ident_n, std::max<int64_t>(scratch_cap_f64(P) / 2, 1 << 24), kChunkF64);
        ensure_scratch_f64(P, std::max<int64_t>(P.sigma_pl.scratch_elems, 1));
        P.sigma_pl.upload(st);
        P.sigma_fp64_ready = true;
    }
    const int64_t per = std::max<int64_t>(P.sigma_pl.scratch_elems, 1);
    cudaEvent_t e0 = P.take_event(), e1 = P.take_event();
    DMRG_CHECK_CUDA(cudaEventRecord(e0, st));
    for (int v = 0; v < nvec; ++v) {
        DMRG_CHECK_CUDA(cudaMemsetAsync(out + (int64_t)v * P.dim, 0, (size_t)P.dim * 8, st));
        BufTable bt = bond_buffers(P, psi + (int64_t)v * P.dim, out + (int64_t)v * P.dim);
        bt.vstride[BUF_SCR] = per;
        P.sigma_pl.run(bt, 1, st);
    }
    DMRG_CHECK_CUDA(cudaEventRecord(e1, st));
    DMRG_CHECK_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    P.ev_pool.push_back(e0);
    P.ev_pool.push_back(e1);
    P.stats.sigma_acc_calls += nvec;
    P.stats.ms_sigma_acc += ms;
    P.stats.sigma_acc_flops += P.sigma_pl.flops * nvec;
}

void sigma_fp64_units(Plan& P, const double* psi, double* out, int nvec, cudaStream_t st) {
    DMRG_REQUIRE(P.bond > 0, DMRG_EINVAL, "no current bond (call dmrg_set_bond)");
    if (!P.oz) {
        sigma_fp64(P, psi, out, nvec, st);
        return;
    }
    ProductList& pl = P.sigma_units_pl;
    if (!P.sigma_units_ready) {
        pl.clear();
        pl.outs = P.sigma_pl.outs;
        pl.cs = P.sigma_pl.cs;
        pl.tile_m = pl.tile_n = 0;  // 64 x 64 tiles: the FP64 units
        pl.lower(BUF_SCR, BUF_ID, P.ident_n, std::max<int64_t>(scratch_cap_f64(P) / 2, 1 << 24), kChunkF64);
        pl.upload(st);
        P.sigma_units_ready = true;
    }
    ensure_scratch_f64(P, std::max<int64_t>(pl.scratch_elems, 1));
    const int64_t per = std::max<int64_t>(pl.scratch_elems, 1);
    for (int v = 0; v < nvec; ++v) {
        DMRG_CHECK_CUDA(cudaMemsetAsync(out + (int64_t)v * P.dim, 0, (size_t)P.dim * 8, st));
        BufTable bt = bond_buffers(P, psi + (int64_t)v * P.dim, out + (int64_t)v * P.dim);
        bt.vstride[BUF_SCR] = per;
        pl.run(bt, 1, st);
    }
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
}

namespace {
void sigma_body(Plan& P, const double* psi, double* out, int nvec, cudaStream_t st);
}

void sigma(Plan& P, const double* psi, double* out, int nvec, cudaStream_t st) {
    DMRG_REQUIRE(P.bond > 0, DMRG_EINVAL, "no current bond (call dmrg_set_bond)");
    DMRG_REQUIRE(nvec >= 1, DMRG_EINVAL, "nvec must be >= 1");
    if (P.sig_pending.size() >= 64) P.collect_sigma_times(false);
    Plan::SigmaEvents ev{P.take_event(), P.take_event(), P.stats.sigma_flops * nvec,
                         P.mixed() ? (P.stats.sigma_stages[0] + P.stats.sigma_stages[1]) * nvec : 0};
    try {
        DMRG_CHECK_CUDA(cudaEventRecord(ev.a, st));
        sigma_body(P, psi, out, nvec, st);
        DMRG_CHECK_CUDA(cudaEventRecord(ev.b, st));
    } catch (...) {
        P.ev_pool.push_back(ev.a);
        P.ev_pool.push_back(ev.b);
        throw;
    }
    P.sig_pending.push_back(ev);
}

namespace {
void sigma_body(Plan& P, const double* psi, double* out, int nvec, cudaStream_t st) {
    if (!P.mixed()) {
        const int64_t per = std::max<int64_t>(P.sigma_pl.scratch_elems, 1);
        const int group = (int)std::max<int64_t>(1, std::min<int64_t>(nvec, P.n_scratch / per));
        for (int v0 = 0; v0 < nvec; v0 += group) {
            const int nv = std::min(group, nvec - v0);
            DMRG_CHECK_CUDA(cudaMemsetAsync(out + (int64_t)v0 * P.dim, 0, (size_t)nv * P.dim * 8, st));
            BufTable bt = bond_buffers(P, psi + (int64_t)v0 * P.dim, out + (int64_t)v0 * P.dim);
            bt.vstride[BUF_SCR] = per;
            P.sigma_pl.run(bt, nv, st);
        }
        P.stats.sigma_calls += nvec;
        return;
    }
    // mixed precision: bf16 pieces of psi, tensor-core products (TMA-staged), FP64 accumulation of sigma
    ProductList& tl = P.sigma_tc;
    const int G = std::max(1, P.opt.n_roots);
    ensure_psi_pieces(P, (int64_t)G * P.dim_pad);
    // the work of one launch of nv vectors: psi (nv x dim) -> sigma (nv x dim)
    auto enqueue = [&](const double* in, double* o, int nv, cudaStream_t s) {
        for (int v = 0; v < nv; ++v)
            dev_split_blocks(in + (int64_t)v * P.dim, P.d_psi_jobs, P.n_psi_jobs, P.ps_hi + (int64_t)v * P.dim_pad,
                             P.ps_lo + (int64_t)v * P.dim_pad, s,
                             P.nsplit == 3 ? P.ps_lo + P.n_ppc + (int64_t)v * P.dim_pad : nullptr);
        DMRG_CHECK_CUDA(cudaMemsetAsync(o, 0, (size_t)nv * P.dim * 8, s));
        tl.run_tma(sigma_bufs(P, P.bond, o), nv, P.nsplit, s);
    };
    {
        const TcBufs tb = sigma_bufs(P, P.bond, nullptr);
        if (tl.maps.stale(tb)) {
            tl.maps.encode_upload(tb, P.nsplit, st);
            P.drop_graphs();
        }
    }
    tc_prepare(P.nsplit);  // kernel attributes, set outside any capture
    const bool graph = P.opt.sigma_graph != 0;
    if (graph) {
        const int64_t need = 2 * (int64_t)G * P.dim;
        if (need > P.n_sig_io) {
            P.drop_graphs();
            if (P.d_sig_io) P.free(P.d_sig_io, P.n_sig_io);
            P.n_sig_io = need;
            P.d_sig_io = P.alloc(need);
        }
        if (!P.cap_stream) DMRG_CHECK_CUDA(cudaStreamCreateWithFlags(&P.cap_stream, cudaStreamNonBlocking));
    }
    for (int v0 = 0; v0 < nvec; v0 += G) {
        const int nv = std::min(G, nvec - v0);
        if (!graph) {
            enqueue(psi + (int64_t)v0 * P.dim, out + (int64_t)v0 * P.dim, nv, st);
            continue;
        }
        double* gin = P.d_sig_io;
        double* gout = P.d_sig_io + (int64_t)G * P.dim;
        Plan::SigmaGraph& sg = P.sigma_graphs[nv];
        if (!sg.exec) {
            // first use at this bond and vector count: capture on the plan's own stream
            const int64_t l0 = launch_counter();
            cudaGraph_t g = nullptr;
            DMRG_CHECK_CUDA(cudaStreamBeginCapture(P.cap_stream, cudaStreamCaptureModeThreadLocal));
            try {
                enqueue(gin, gout, nv, P.cap_stream);
            } catch (...) {
                cudaStreamEndCapture(P.cap_stream, &g);
                if (g) cudaGraphDestroy(g);
                throw;
            }
            DMRG_CHECK_CUDA(cudaStreamEndCapture(P.cap_stream, &g));
            DMRG_CHECK_CUDA(cudaGraphInstantiate(&sg.exec, g, 0));
            cudaGraphDestroy(g);
            sg.launches = launch_counter() - l0;
            launch_counter() = l0;
        }
        DMRG_CHECK_CUDA(cudaMemcpyAsync(gin, psi + (int64_t)v0 * P.dim, (size_t)nv * P.dim * 8,
                                        cudaMemcpyDeviceToDevice, st));
        DMRG_CHECK_CUDA(cudaGraphLaunch(sg.exec, st));
        launch_counter() += sg.launches;
        DMRG_CHECK_CUDA(cudaMemcpyAsync(out + (int64_t)v0 * P.dim, gout, (size_t)nv * P.dim * 8,
                                        cudaMemcpyDeviceToDevice, st));
    }
    P.stats.sigma_calls += nvec;
    P.check_device_error();
}
}  // namespace

void hdiag(Plan& P, double* out, cudaStream_t st) {
    DMRG_REQUIRE(P.bond > 0, DMRG_EINVAL, "no current bond (call dmrg_set_bond)");
    BufTable bt = bond_buffers(P, nullptr, out);
    cudaEvent_t e0 = P.take_event(), e1 = P.take_event();
    DMRG_CHECK_CUDA(cudaEventRecord(e0, st));
    P.hdiag_pl.run(bt, 1, st);
    DMRG_CHECK_CUDA(cudaEventRecord(e1, st));
    DMRG_CHECK_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    DMRG_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    P.stats.ms_hdiag += ms;
    P.ev_pool.push_back(e0);
    P.ev_pool.push_back(e1);
}

}  // namespace dmrg

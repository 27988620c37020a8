// C-ABI of libdmrg (declared in include/dmrg.h).  Every entry point catches
// exceptions and returns a status code; nothing aborts.
#include <cmath>
#include <cstring>
#include <mutex>

#include "bond.h"
#include "tc.h"

using namespace dmrg;

struct dmrg_plan_s {
    Plan P;
};

namespace {
std::string g_last_error;
std::mutex g_err_mu;

dmrg_status fail(dmrg_plan_t plan, dmrg_status code, const std::string& msg) {
    if (plan) plan->P.last_error = msg;
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_last_error = msg;
    return code;
}

template <class F>
dmrg_status guarded(dmrg_plan_t plan, F&& f) {
    try {
        return f();
    } catch (const Error& e) {
        return fail(plan, e.code, e.what());
    } catch (const std::exception& e) {
        return fail(plan, DMRG_EINVAL, e.what());
    }
}

// Tensor-core grouped GEMM on FP64 operand buffers: the operands are split
// into bf16 pieces on the device, the product runs on tcgen05, and C is
// accumulated in FP64.  Leading dimensions and offsets must be multiples of
// 8 elements; segment alphas must be +1 or -1, except for single-segment
// blocks (scaled in the epilogue).
dmrg_status grouped_gemm_tc(int nsplit, int n_out, const int* m, const int* n, const int64_t* c_off,
                            const int* seg_beg, const int* k, const int64_t* a_off, const int* lda,
                            const int* a_tr, const int64_t* b_off, const int* ldb, const int* b_tr,
                            const double* alpha, const double* a, const double* b, double* c,
                            cudaStream_t st) {
    int64_t ea = 8, eb = 8, ec = 0;
    WorkList wl;
    for (int o = 0; o < n_out; ++o) {
        DMRG_REQUIRE(m[o] >= 0 && n[o] >= 0 && c_off[o] >= 0, DMRG_EINVAL, "bad block size");
        ec = std::max<int64_t>(ec, c_off[o] + (int64_t)m[o] * n[o]);
        std::vector<Seg> segs;
        const int ns = seg_beg[o + 1] - seg_beg[o];
        float tile_alpha = 1.0f;
        for (int s = seg_beg[o]; s < seg_beg[o + 1]; ++s) {
            DMRG_REQUIRE(k[s] >= 0 && lda[s] >= 1 && ldb[s] >= 1, DMRG_EINVAL, "bad segment");
            DMRG_REQUIRE(lda[s] % 8 == 0 && ldb[s] % 8 == 0 && a_off[s] % 8 == 0 && b_off[s] % 8 == 0, DMRG_EINVAL,
                         "tensor-core operands need 8-element aligned offsets and leading dimensions");
            Seg g{};
            g.a_off = a_off[s];
            g.b_off = b_off[s];
            g.k = k[s];
            g.lda = lda[s];
            g.ldb = ldb[s];
            g.a_tr = (uint8_t)(a_tr[s] != 0);
            g.b_tr = (uint8_t)(b_tr[s] != 0);
            g.a_buf = 0;
            g.b_buf = 1;
            if (ns == 1) {
                tile_alpha = (float)alpha[s];
                g.alpha = 1.0;
            } else {
                DMRG_REQUIRE(alpha[s] == 1.0 || alpha[s] == -1.0, DMRG_EINVAL, "segment alpha must be +-1");
                g.alpha = alpha[s];
            }
            // extents of the operands read
            const int64_t ar = g.a_tr ? g.k : m[o], ac = g.a_tr ? m[o] : g.k;
            const int64_t br = g.b_tr ? n[o] : g.k, bc = g.b_tr ? g.k : n[o];
            if (ar > 0 && ac > 0) ea = std::max<int64_t>(ea, g.a_off + (ar - 1) * g.lda + ac);
            if (br > 0 && bc > 0) eb = std::max<int64_t>(eb, g.b_off + (br - 1) * g.ldb + bc);
            segs.push_back(g);
        }
        wl.add_block(c_off[o], 2, m[o], n[o], n[o], segs, TC_ATOMIC_F64, 1024, 128, tile_alpha);
    }
    const int64_t ea_n = ea, eb_n = eb;  // elements actually present in a / b
    ea = round_up(ea, 8);
    eb = round_up(eb, 8);
    __nv_bfloat16 *ha = nullptr, *la = nullptr, *hb = nullptr, *lb = nullptr;
    int* ctr = nullptr;
    const int lop = nsplit == 3 ? 2 : 1;  // pieces held in the lo arrays
    DMRG_CHECK_CUDA(cudaMalloc(&ha, ea * 2));
    DMRG_CHECK_CUDA(cudaMalloc(&la, lop * ea * 2));
    DMRG_CHECK_CUDA(cudaMalloc(&hb, eb * 2));
    DMRG_CHECK_CUDA(cudaMalloc(&lb, lop * eb * 2));
    DMRG_CHECK_CUDA(cudaMalloc(&ctr, 2 * sizeof(int)));
    DMRG_CHECK_CUDA(cudaMemsetAsync(ctr, 0, 2 * sizeof(int), st));
    DMRG_REQUIRE(ea < 2147483647 && eb < 2147483647, DMRG_EINVAL, "operand too large");
    dev_split_f64(a, 1, (int)ea_n, ea_n, ha, la, ea, st, nsplit == 3 ? la + ea : nullptr);
    dev_split_f64(b, 1, (int)eb_n, eb_n, hb, lb, eb, st, nsplit == 3 ? lb + eb : nullptr);
    if (ec > 0) DMRG_CHECK_CUDA(cudaMemsetAsync(c, 0, ec * 8, st));
    wl.upload(st);
    TcBufs tb{};
    tb.hi[0] = ha;
    tb.lo[0] = la;
    tb.hi[1] = hb;
    tb.lo[1] = lb;
    if (nsplit == 3) {
        tb.pstride[0] = ea;
        tb.pstride[1] = eb;
    }
    tb.out[2] = c;
    tb.counter = ctr;
    tb.err = ctr + 1;
    launch_seg_gemm_tc(wl, tb, 1, nsplit, st);
    int err = 0;
    DMRG_CHECK_CUDA(cudaMemcpyAsync(&err, ctr + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    wl.release();
    cudaFree(ha);
    cudaFree(la);
    cudaFree(hb);
    cudaFree(lb);
    cudaFree(ctr);
    if (err) return fail(nullptr, DMRG_ETIMEOUT, "tensor-core kernel wait timed out");
    return DMRG_OK;
}

cudaStream_t pick(dmrg_plan_t plan, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    plan->P.stream = s;
    return s;
}

}  // namespace

extern "C" {

void dmrg_default_options(dmrg_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = DMRG_FP64;
    o->n_roots = 1;
    o->tol = 1e-6;
    o->max_iter = 200;
    o->max_space = 0;
    o->precond = DMRG_PRECOND_JACOBI;
    o->fp64_final = 0;
    o->mem_budget = 0;
    o->scratch_bytes = 0;
    o->keep_envs = 0;
    o->verbose = 0;
    o->tc_kchunk = 0;
    o->fp64_store = 0;
    o->sigma_graph = 1;
    o->sigma_tune = 1;
    o->sigma_tile_n = 0;
    o->refine = 0;
    o->max_refine = 0;
    o->fp64_tc = 0;
    o->host_tier = 0;
    o->sigma_per_term = 0;
    o->decim_tol32 = 0.0;
    o->decim_fp64_units = 0;
}

const char* dmrg_version(void) {
    return "libdmrg 0.2 (sm_103a; FP64 segmented grouped GEMM; tcgen05 bf16-piece engine)";
}

dmrg_status dmrg_plan(const double* h, const double* chol, int n_chol, double e_core, int K, int N, int twoS,
                      int D, const dmrg_options* opt, const char* mps_path, dmrg_plan_t* out) {
    if (!out) return fail(nullptr, DMRG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!h || !chol || n_chol < 0 || K < 2 || K > 512 || N < 0 || N > 2 * K || D < 1)
        return fail(nullptr, DMRG_EINVAL, "bad sizes");
    if (n_chol == 0 && K > 128) return fail(nullptr, DMRG_EINVAL, "a full (pq|rs) array is accepted up to K = 128");
    if (((N + twoS) & 1) || std::abs(twoS) > std::min(N, 2 * K - N))
        return fail(nullptr, DMRG_EINVAL, "inconsistent N / 2Sz");
    if (!mps_path) return fail(nullptr, DMRG_EINVAL, "an MPS file is required");
    for (int64_t i = 0; i < (int64_t)K * K; ++i)
        if (!std::isfinite(h[i])) return fail(nullptr, DMRG_ENUMERIC, "non-finite one-electron integral");
    const int64_t n_in = n_chol > 0 ? (int64_t)n_chol * K * K : (int64_t)K * K * K * K;
    for (int64_t i = 0; i < n_in; ++i)
        if (!std::isfinite(chol[i]))
            return fail(nullptr, DMRG_ENUMERIC, n_chol > 0 ? "non-finite Cholesky vector" : "non-finite (pq|rs)");
    if (n_chol == 0) {
        // real orbitals: (pq|rs) = (qp|rs) = (pq|sr) = (rs|pq)
        const int64_t K2 = (int64_t)K * K;
        double amax = 0.0, dmax = 0.0;
        for (int64_t i = 0; i < K2 * K2; ++i) amax = std::max(amax, std::fabs(chol[i]));
        for (int p = 0; p < K; ++p)
            for (int q = 0; q < K; ++q)
                for (int r = 0; r < K; ++r)
                    for (int t = 0; t < K; ++t) {
                        const double x = chol[((int64_t)p * K + q) * K2 + r * K + t];
                        dmax = std::max(dmax, std::fabs(x - chol[((int64_t)q * K + p) * K2 + r * K + t]));
                        dmax = std::max(dmax, std::fabs(x - chol[((int64_t)p * K + q) * K2 + t * K + r]));
                        dmax = std::max(dmax, std::fabs(x - chol[((int64_t)r * K + t) * K2 + p * K + q]));
                    }
        if (dmax > 1e-12 * std::max(amax, 1.0))
            return fail(nullptr, DMRG_EINVAL, "(pq|rs) lacks the symmetry of real orbitals");
    }
    auto* plan = new dmrg_plan_s();
    dmrg_status st = guarded(plan, [&]() -> dmrg_status {
        Plan& P = plan->P;
        if (opt) P.opt = *opt;
        else dmrg_default_options(&P.opt);
        if (P.opt.precision == DMRG_FP64) P.nsplit = 0;
        else if (P.opt.precision == DMRG_BF16X3) P.nsplit = 2;
        else if (P.opt.precision == DMRG_BF16) P.nsplit = 1;
        else if (P.opt.precision == DMRG_BF16X6) P.nsplit = 3;
        else if (P.opt.precision == DMRG_FP64_TC) P.nsplit = 0;
        else throw Error(DMRG_EINVAL, "unknown precision mode");
        // FP64 products on the tensor-core engine: the FP64_TC mode, or the FP64
        // store of a mixed mode with fp64_tc
        P.oz = P.opt.precision == DMRG_FP64_TC || (P.nsplit > 0 && P.opt.fp64_store && P.opt.fp64_tc);
        if (P.opt.sigma_tile_n != 0 && P.opt.sigma_tile_n != 64 && P.opt.sigma_tile_n != 128)
            throw Error(DMRG_EINVAL, "sigma_tile_n must be 0, 64 or 128");
        P.K = K;
        P.N = N;
        P.twoS = twoS;
        P.D = D;
        P.n_so = 2 * K;
        P.tot = QN(N, twoS);
        P.I.K = K;
        P.I.e_core = e_core;
        P.I.h.assign(h, h + (int64_t)K * K);
        std::string err;
        if (!P.mps.read(mps_path, err)) throw Error(DMRG_EIO, err);
        if (P.mps.K != K || P.mps.N != N || P.mps.twoS != twoS)
            throw Error(DMRG_EINVAL, "MPS file does not match K / N / 2Sz");
        if (P.mps.bonds[0].size() != 1 || P.mps.bonds[K].size() != 1 || P.mps.bonds[K][0][0] != N ||
            P.mps.bonds[K][0][1] != twoS)
            throw Error(DMRG_EINVAL, "MPS boundary sectors do not match the quantum numbers");
        size_t freeb = 0, totb = 0;
        DMRG_CHECK_CUDA(cudaMemGetInfo(&freeb, &totb));
        P.budget = P.opt.mem_budget > 0 ? P.opt.mem_budget : (int64_t)(0.9 * (double)freeb);
        const int64_t K2 = (int64_t)K * K;
        P.left.resize(K + 1);
        P.right.resize(K + 1);
        if (n_chol == 0) {  // the full array as given
            P.I.eri.assign(chol, chol + K2 * K2);
            return DMRG_OK;
        }
        // (pq|rs) = sum_X L[X][pq] L[X][rs] on the device
        double* dL = P.alloc(n_chol * K2);
        double* dE = P.alloc(K2 * K2);
        DMRG_CHECK_CUDA(cudaMemcpy(dL, chol, n_chol * K2 * 8, cudaMemcpyHostToDevice));
        WorkList wl;
        Seg s{};
        s.a_off = 0;
        s.lda = (int)K2;
        s.a_tr = 1;  // A(pq, X) = L[X][pq]
        s.b_off = 0;
        s.ldb = (int)K2;
        s.b_tr = 0;  // B(X, rs) = L[X][rs]
        s.k = n_chol;
        s.a_buf = 0;
        s.b_buf = 0;
        s.alpha = 1.0;
        wl.add_block(0, 1, (int)K2, (int)K2, (int)K2, {s}, TILE_STORE);
        wl.upload(nullptr);
        BufTable bt{};
        bt.p[0] = dL;
        bt.p[1] = dE;
        launch_seg_gemm_f64(wl, bt, 1, nullptr);
        P.I.eri.resize(K2 * K2);
        DMRG_CHECK_CUDA(cudaMemcpy(P.I.eri.data(), dE, K2 * K2 * 8, cudaMemcpyDeviceToHost));
        wl.release();
        P.free(dL, n_chol * K2);
        P.free(dE, K2 * K2);
        return DMRG_OK;
    });
    if (st != DMRG_OK) {
        delete plan;
        return st;
    }
    *out = plan;
    return DMRG_OK;
}

dmrg_status dmrg_set_bond(dmrg_plan_t plan, int k, void* stream) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    return guarded(plan, [&]() {
        pick(plan, stream);
        set_bond(plan->P, k);
        return DMRG_OK;
    });
}

dmrg_status dmrg_layout(dmrg_plan_t plan, int64_t* dim, int* n_sectors, int64_t* offsets, int* qn) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    Plan& P = plan->P;
    if (P.bond < 1) return fail(plan, DMRG_EINVAL, "no current bond");
    if (dim) *dim = P.dim;
    if (n_sectors) *n_sectors = (int)P.layout.size();
    const auto& bl = P.mps.bonds[P.bond - 1];
    for (size_t i = 0; i < P.layout.size(); ++i) {
        const Plan::Sector& s = P.layout[i];
        if (offsets) offsets[i] = s.off;
        if (qn) {
            qn[6 * i + 0] = bl[s.il][0];
            qn[6 * i + 1] = bl[s.il][1];
            qn[6 * i + 2] = s.y / 4;
            qn[6 * i + 3] = s.y % 4;
            qn[6 * i + 4] = s.dl;
            qn[6 * i + 5] = s.dr;
        }
    }
    if (offsets) offsets[P.layout.size()] = P.dim;
    return DMRG_OK;
}

dmrg_status dmrg_sigma(dmrg_plan_t plan, const double* psi, double* sig, int nvec, void* stream) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    if (!psi || !sig) return fail(plan, DMRG_EINVAL, "NULL vector");
    return guarded(plan, [&]() {
        cudaStream_t st = pick(plan, stream);
        Plan& P = plan->P;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
        sigma(P, psi, sig, nvec, st);
        cudaEventRecord(e1, st);
        DMRG_CHECK_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        P.stats.sigma_ms_last = ms;
        P.stats.ms_gemm += ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return DMRG_OK;
    });
}

dmrg_status dmrg_sigma_fp64(dmrg_plan_t plan, const double* psi, double* sig, int nvec, void* stream) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    if (!psi || !sig || nvec < 1) return fail(plan, DMRG_EINVAL, "bad arguments");
    return guarded(plan, [&]() {
        cudaStream_t st = pick(plan, stream);
        sigma_fp64(plan->P, psi, sig, nvec, st);
        DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
        return DMRG_OK;
    });
}

dmrg_status dmrg_sigma_fp64_units(dmrg_plan_t plan, const double* psi, double* sig, int nvec, void* stream) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    if (!psi || !sig || nvec < 1) return fail(plan, DMRG_EINVAL, "bad arguments");
    return guarded(plan, [&]() {
        cudaStream_t st = pick(plan, stream);
        sigma_fp64_units(plan->P, psi, sig, nvec, st);
        return DMRG_OK;
    });
}

dmrg_status dmrg_sigma_host(dmrg_plan_t plan, const double* psi, double* sig, int nvec, void* stream) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    if (!psi || !sig || nvec < 1) return fail(plan, DMRG_EINVAL, "bad arguments");
    return guarded(plan, [&]() {
        cudaStream_t st = pick(plan, stream);
        Plan& P = plan->P;
        DMRG_REQUIRE(P.bond > 0, DMRG_EINVAL, "no current bond");
        int64_t need = 2 * (int64_t)nvec * P.dim;
        if (need > P.n_io) {
            P.free(P.d_io, P.n_io);
            P.n_io = need;
            P.d_io = P.alloc(need);
        }
        double* dpsi = P.d_io;
        double* dsig = P.d_io + (int64_t)nvec * P.dim;
        DMRG_CHECK_CUDA(cudaMemcpyAsync(dpsi, psi, (size_t)nvec * P.dim * 8, cudaMemcpyHostToDevice, st));
        sigma(P, dpsi, dsig, nvec, st);
        DMRG_CHECK_CUDA(cudaMemcpyAsync(sig, dsig, (size_t)nvec * P.dim * 8, cudaMemcpyDeviceToHost, st));
        DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
        return DMRG_OK;
    });
}

dmrg_status dmrg_hdiag(dmrg_plan_t plan, double* diag, void* stream) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    if (!diag) return fail(plan, DMRG_EINVAL, "NULL vector");
    return guarded(plan, [&]() {
        cudaStream_t st = pick(plan, stream);
        hdiag(plan->P, diag, st);
        DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
        return DMRG_OK;
    });
}

dmrg_status dmrg_davidson(dmrg_plan_t plan, double* psi, int n_roots, double tol, int max_iter, int precond,
                          double* energies, int* iters, void* stream) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    if (!psi || !energies || tol <= 0 || max_iter < 1) return fail(plan, DMRG_EINVAL, "bad arguments");
    return guarded(plan, [&]() {
        pick(plan, stream);
        return davidson(plan->P, psi, n_roots, tol, max_iter, precond, energies, iters);
    });
}

dmrg_status dmrg_mlp_init(dmrg_plan_t plan, uint32_t seed) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    return guarded(plan, [&]() {
        Plan& P = plan->P;
        mlp_init(P.mlp, seed, P.stream);
        DMRG_CHECK_CUDA(cudaStreamSynchronize(P.stream));
        P.mlp.trained = false;
        return DMRG_OK;
    });
}

dmrg_status dmrg_mlp_harvest(dmrg_plan_t plan, double* psi, int max_iter, int jd_iters, int64_t per_solve,
                             double* energy, int64_t* n_pairs, void* stream) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    if (!psi || max_iter < 1 || jd_iters < 1 || per_solve < 1) return fail(plan, DMRG_EINVAL, "bad arguments");
    return guarded(plan, [&]() {
        pick(plan, stream);
        Plan& P = plan->P;
        if (!P.mlp.d_w) mlp_init(P.mlp, 3u, P.stream);
        P.harvest.on = true;
        P.harvest.jd_iters = jd_iters;
        P.harvest.per_solve = per_solve;
        const int64_t before = P.harvest.pairs;
        double e = 0.0;
        int it = 0;
        dmrg_status st = DMRG_OK;
        try {
            st = davidson(P, psi, 1, P.opt.tol, max_iter, DMRG_PRECOND_JACOBI, &e, &it);
        } catch (...) {
            P.harvest.on = false;
            throw;
        }
        P.harvest.on = false;
        if (energy) *energy = e;
        if (n_pairs) *n_pairs = P.harvest.pairs - before;
        return st == DMRG_ENOTCONV ? DMRG_OK : st;
    });
}

dmrg_status dmrg_mlp_train(dmrg_plan_t plan, int steps, int64_t batch, float lr, uint64_t seed, float* loss_first,
                           float* loss_last, float* held_first, float* held_last, void* stream) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    if (steps < 1 || batch < 1 || !(lr > 0.f)) return fail(plan, DMRG_EINVAL, "bad arguments");
    return guarded(plan, [&]() {
        cudaStream_t st = pick(plan, stream);
        Plan& P = plan->P;
        if (!P.mlp.d_w) mlp_init(P.mlp, 3u, st);
        mlp_train(P.mlp, steps, batch, lr, seed, loss_first, loss_last, held_first, held_last, st);
        return DMRG_OK;
    });
}

dmrg_status dmrg_mlp_eval(dmrg_plan_t plan, const float* x, int64_t n, float* g, int bf16, void* stream) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    if (!x || !g || n < 0) return fail(plan, DMRG_EINVAL, "bad arguments");
    return guarded(plan, [&]() {
        cudaStream_t st = pick(plan, stream);
        Plan& P = plan->P;
        DMRG_REQUIRE(P.mlp.d_w, DMRG_EINVAL, "MLP not initialised (dmrg_mlp_init)");
        mlp_forward(P.mlp, x, n, g, bf16 != 0, st);
        DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
        return DMRG_OK;
    });
}

dmrg_status dmrg_mlp_gradient(dmrg_plan_t plan, const float* x, const float* y, const float* w, int64_t n,
                              float* grad, float* loss, void* stream) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    if (!x || !y || !grad || !loss || n < 1) return fail(plan, DMRG_EINVAL, "bad arguments");
    return guarded(plan, [&]() {
        cudaStream_t st = pick(plan, stream);
        Plan& P = plan->P;
        DMRG_REQUIRE(P.mlp.d_w, DMRG_EINVAL, "MLP not initialised (dmrg_mlp_init)");
        mlp_gradient(P.mlp, x, y, w, n, grad, loss, st);
        DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
        return DMRG_OK;
    });
}

dmrg_status dmrg_mlp_params(dmrg_plan_t plan, float* host, int set) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    if (!host) return fail(plan, DMRG_EINVAL, "bad arguments");
    return guarded(plan, [&]() {
        Plan& P = plan->P;
        if (!P.mlp.d_w) mlp_init(P.mlp, 3u, P.stream);
        if (set) {
            DMRG_CHECK_CUDA(cudaMemcpyAsync(P.mlp.d_w, host, kMlpParams * sizeof(float), cudaMemcpyHostToDevice,
                                            P.stream));
            mlp_publish(P.mlp, P.stream);
            P.mlp.trained = true;
        } else {
            DMRG_CHECK_CUDA(cudaMemcpyAsync(host, P.mlp.d_w, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost,
                                            P.stream));
        }
        DMRG_CHECK_CUDA(cudaStreamSynchronize(P.stream));
        return DMRG_OK;
    });
}

int dmrg_mlp_num_params(void) { return kMlpParams; }

dmrg_status dmrg_decimate(dmrg_plan_t plan, const double* psi, int n_roots, int D, int forward, double* discarded,
                          double* next_psi, int64_t* next_dim, void* stream) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    if (!psi || n_roots < 1 || D < 1) return fail(plan, DMRG_EINVAL, "bad arguments");
    return guarded(plan, [&]() {
        cudaStream_t st = pick(plan, stream);
        Plan& P = plan->P;
        int64_t cap = next_dim ? *next_dim : 0;
        decimate(P, psi, n_roots, D, forward != 0, discarded);
        if (next_dim) *next_dim = P.dim;
        if (next_psi && cap >= P.dim)
            DMRG_CHECK_CUDA(cudaMemcpyAsync(next_psi, P.d_guess, (size_t)n_roots * P.dim * 8,
                                            cudaMemcpyDeviceToDevice, st));
        DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
        return DMRG_OK;
    });
}

dmrg_status dmrg_set_refine(dmrg_plan_t plan, int refine, int max_refine) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    if (max_refine < 0) return fail(plan, DMRG_EINVAL, "max_refine must be >= 0");
    plan->P.opt.refine = refine != 0;
    plan->P.opt.max_refine = max_refine;
    return DMRG_OK;
}

dmrg_status dmrg_update_bond_host(dmrg_plan_t plan, const double* psi_host, int n_roots, int D, int forward,
                                  double* energies, int* iters, double* discarded, double* next_psi_host,
                                  int64_t* next_dim, void* stream) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    if (!psi_host || !energies || n_roots < 1 || D < 1 || (next_psi_host && !next_dim))
        return fail(plan, DMRG_EINVAL, "bad arguments");
    return guarded(plan, [&]() {
        cudaStream_t st = pick(plan, stream);
        Plan& P = plan->P;
        DMRG_REQUIRE(P.bond > 0, DMRG_EINVAL, "no current bond");
        const int64_t need = (int64_t)n_roots * P.dim;
        if (need > P.n_io) {
            P.free(P.d_io, P.n_io);
            P.n_io = need;
            P.d_io = P.alloc(need);
        }
        double* dpsi = P.d_io;
        DMRG_CHECK_CUDA(cudaMemcpyAsync(dpsi, psi_host, (size_t)need * 8, cudaMemcpyHostToDevice, st));
        const dmrg_status ds = davidson(P, dpsi, n_roots, P.opt.tol, P.opt.max_iter, P.opt.precond, energies, iters);
        const int64_t cap = next_dim ? *next_dim : 0;
        double w = 0.0;
        decimate(P, dpsi, n_roots, D, forward != 0, &w);
        if (discarded) *discarded = w;
        if (next_dim) *next_dim = P.dim;
        if (next_psi_host && cap >= P.dim)
            DMRG_CHECK_CUDA(cudaMemcpyAsync(next_psi_host, P.d_guess, (size_t)n_roots * P.dim * 8,
                                            cudaMemcpyDeviceToHost, st));
        DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
        return ds;
    });
}

dmrg_status dmrg_sweep(dmrg_plan_t plan, int n_sweeps, const int* D_schedule, double* energies, double* discarded,
                       void* stream) {
    if (!plan) return fail(nullptr, DMRG_EINVAL, "plan is NULL");
    if (n_sweeps < 1 || !energies) return fail(plan, DMRG_EINVAL, "bad arguments");
    return guarded(plan, [&]() {
        pick(plan, stream);
        return sweep(plan->P, n_sweeps, D_schedule, energies, discarded);
    });
}

dmrg_status dmrg_extrapolate(const double* w, const double* E, int n, double* e0, double* slope, double* rms) {
    if (!w || !E || !e0 || n < 2) return fail(nullptr, DMRG_EINVAL, "extrapolation needs two points and outputs");
    // centred two-pass least squares: mean, then the centred moments
    double mw = 0.0, mE = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!std::isfinite(w[i]) || !std::isfinite(E[i]))
            return fail(nullptr, DMRG_EINVAL, "non-finite point in the extrapolation series");
        mw += w[i];
        mE += E[i];
    }
    mw /= n;
    mE /= n;
    double sxx = 0.0, sxy = 0.0;
    for (int i = 0; i < n; ++i) {
        sxx += (w[i] - mw) * (w[i] - mw);
        sxy += (w[i] - mw) * (E[i] - mE);
    }
    if (!(sxx > 0.0)) return fail(nullptr, DMRG_EINVAL, "all discarded weights are equal");
    const double a = sxy / sxx;
    const double b = mE - a * mw;
    *e0 = b;
    if (slope) *slope = a;
    if (rms) {
        double r2 = 0.0;
        for (int i = 0; i < n; ++i) {
            const double r = E[i] - (a * w[i] + b);
            r2 += r * r;
        }
        *rms = std::sqrt(r2 / n);
    }
    return DMRG_OK;
}

dmrg_status dmrg_save_mps(dmrg_plan_t plan, const char* path) {
    if (!plan || !path) return fail(plan, DMRG_EINVAL, "bad arguments");
    if (!plan->P.mps.write(path)) return fail(plan, DMRG_EIO, std::string("cannot write ") + path);
    return DMRG_OK;
}

dmrg_status dmrg_stats(dmrg_plan_t plan, dmrg_stats_t* out) {
    if (!plan || !out) return fail(plan, DMRG_EINVAL, "bad arguments");
    return guarded(plan, [&]() {
        plan->P.collect_sigma_times(true);
        plan->P.stats.kernel_launches = launch_counter();
        plan->P.stats.device_bytes = plan->P.dev_bytes;
        *out = plan->P.stats;
        return DMRG_OK;
    });
}

const char* dmrg_last_error(dmrg_plan_t plan) {
    if (plan) return plan->P.last_error.c_str();
    return g_last_error.c_str();
}

void dmrg_destroy(dmrg_plan_t plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    delete plan;
}

dmrg_status dmrg_grouped_gemm(int precision, int n_out, const int* m, const int* n, const int64_t* c_off,
                              const int* seg_beg, const int* k, const int64_t* a_off, const int* lda, const int* a_tr,
                              const int64_t* b_off, const int* ldb, const int* b_tr, const double* alpha,
                              const double* a, const double* b, double* c, void* stream) {
    if (n_out < 0 || !m || !n || !c_off || !seg_beg || !a || !b || !c) return fail(nullptr, DMRG_EINVAL, "bad arguments");
    if (precision != DMRG_FP64 && precision != DMRG_BF16X3 && precision != DMRG_BF16 && precision != DMRG_BF16X6 &&
        precision != DMRG_FP64_TC)
        return fail(nullptr, DMRG_EINVAL, "unknown precision");
    if (precision != DMRG_FP64 && precision != DMRG_FP64_TC) {
        try {
            return grouped_gemm_tc(precision == DMRG_BF16X3 ? 2 : (precision == DMRG_BF16X6 ? 3 : 1), n_out, m, n, c_off, seg_beg, k, a_off, lda, a_tr,
                                   b_off, ldb, b_tr, alpha, a, b, c, (cudaStream_t)stream);
        } catch (const Error& e) {
            return fail(nullptr, e.code, e.what());
        }
    }
    try {
        cudaStream_t st = (cudaStream_t)stream;
        WorkList wl;
        if (precision == DMRG_FP64_TC) {  // 128 x 64 tiles: the FP64-accurate tensor-core engine
            wl.tile_m = oz_tile_rows();
            wl.tile_n = oz_tile_cols();
        }
        for (int o = 0; o < n_out; ++o) {
            std::vector<Seg> segs;
            for (int s = seg_beg[o]; s < seg_beg[o + 1]; ++s) {
                Seg g{};
                g.a_off = a_off[s];
                g.b_off = b_off[s];
                g.k = k[s];
                g.lda = lda[s];
                g.ldb = ldb[s];
                g.a_tr = (uint8_t)(a_tr[s] != 0);
                g.b_tr = (uint8_t)(b_tr[s] != 0);
                g.a_buf = 0;
                g.b_buf = 1;
                g.alpha = alpha[s];
                if (g.k < 0 || g.lda < 1 || g.ldb < 1) return fail(nullptr, DMRG_EINVAL, "bad segment");
                segs.push_back(g);
            }
            if (m[o] < 0 || n[o] < 0) return fail(nullptr, DMRG_EINVAL, "bad block size");
            wl.add_block(c_off[o], 2, m[o], n[o], n[o], segs, TILE_STORE);
        }
        wl.upload(st);
        BufTable bt{};
        bt.p[0] = const_cast<double*>(a);
        bt.p[1] = const_cast<double*>(b);
        bt.p[2] = c;
        launch_seg_gemm_f64(wl, bt, 1, st);
        DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
        wl.release();
        if (precision == DMRG_FP64_TC && oz_take_error(st))
            return fail(nullptr, DMRG_ETIMEOUT, "the FP64 tensor-core engine gave up waiting");
        return DMRG_OK;
    } catch (const Error& e) {
        return fail(nullptr, e.code, e.what());
    }
}

dmrg_status dmrg_grouped_gemm_noalloc(int n_out, const int* m, const int* n, const int64_t* c_off, const int* seg_beg,
                                      const int* k, const int64_t* a_off, const int* lda, const int* a_tr,
                                      const int64_t* b_off, const int* ldb, const int* b_tr, const double* alpha,
                                      const double* a, const double* b, double* c, void* stream) {
    if (n_out < 0 || !m || !n || !c_off || !seg_beg || !a || !b || !c) return fail(nullptr, DMRG_EINVAL, "bad arguments");
    try {
        WorkList wl;
        for (int o = 0; o < n_out; ++o) {
            if (m[o] < 0 || n[o] < 0 || c_off[o] < 0) return fail(nullptr, DMRG_EINVAL, "bad block size");
            std::vector<Seg> segs;
            for (int s = seg_beg[o]; s < seg_beg[o + 1]; ++s) {
                Seg g{};
                g.a_off = a_off[s];
                g.b_off = b_off[s];
                g.k = k[s];
                g.lda = lda[s];
                g.ldb = ldb[s];
                g.a_tr = (uint8_t)(a_tr[s] != 0);
                g.b_tr = (uint8_t)(b_tr[s] != 0);
                g.a_buf = 0;
                g.b_buf = 1;
                g.alpha = alpha[s];
                if (g.k < 0 || g.lda < 1 || g.ldb < 1) return fail(nullptr, DMRG_EINVAL, "bad segment");
                segs.push_back(g);
            }
            wl.add_block(c_off[o], 2, m[o], n[o], n[o], segs, TILE_STORE);
        }
        grouped_gemm_f64_noalloc(wl, a, b, c, (cudaStream_t)stream);
        return DMRG_OK;
    } catch (const Error& e) {
        return fail(nullptr, e.code, e.what());
    }
}

int64_t dmrg_noalloc_scratch_bytes(void) { return noalloc_scratch_bytes(); }

dmrg_status dmrg_selftest_wait(double seconds, int arrive, void* stream) {
    if (!(seconds > 0.0 && seconds <= 2.0)) return fail(nullptr, DMRG_EINVAL, "seconds must lie in (0, 2]");
    try {
        if (wait_selftest(seconds, arrive != 0, (cudaStream_t)stream)) return DMRG_OK;
        return fail(nullptr, DMRG_ETIMEOUT, "bounded device wait gave up (self-test)");
    } catch (const Error& e) {
        return fail(nullptr, e.code, e.what());
    }
}

}  // extern "C"

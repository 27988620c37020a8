// Davidson eigensolver (Sec. 2.1, Davidson 1975), decimation by the
// (state-averaged) reduced density matrix (Sec. 2.1), and the two-dot sweep
// (Sec. 2.3, Fig. flowchart).  All vector arithmetic runs on the device in
// FP64; the host keeps only the small subspace matrix and scalars.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>

#include "bond.h"
#include "eig.h"
#include "mlp.h"

namespace dmrg {

namespace {
enum : int8_t { BUF_L = 0, BUF_R = 1, BUF_INT = 2, BUF_PSI = 3, BUF_SCR = 4, BUF_ID = 5, BUF_OUT = 6, BUF_W = 7 };

double host_dot(Plan& P, const double* x, const double* y, int64_t n, double* d_out, double* d_work) {
    dev_dots(x, n, 1, y, n, d_out, d_work, P.stream);
    double r = 0.0;
    DMRG_CHECK_CUDA(cudaMemcpyAsync(&r, d_out, 8, cudaMemcpyDeviceToHost, P.stream));
    DMRG_CHECK_CUDA(cudaStreamSynchronize(P.stream));
    return r;
}
}  // namespace

// ---------------------------------------------------------------------------
// Jacobi-Davidson correction equation (training pairs of the learned
// preconditioner): (I - u u^T)(H - theta)(I - u u^T) t = -r, t orthogonal to u,
// solved by MINRES (Paige and Saunders, 1975) with the plan's sigma.
// ---------------------------------------------------------------------------

namespace {

int jd_solve(Plan& P, const double* u, double theta, const double* r, double* t, int max_it, double tol,
             double* dco, double* dwork) {
    const int64_t n = P.dim;
    cudaStream_t st = P.stream;
    double* buf = P.alloc(7 * n);
    double *r1 = buf, *r2 = buf + n, *y = buf + 2 * n, *v = buf + 3 * n, *w = buf + 4 * n, *w1 = buf + 5 * n,
           *w2 = buf + 6 * n;
    auto dot = [&](const double* a, const double* b) { return host_dot(P, a, b, n, dco, dwork); };
    // b = -r
    dev_axpby(-1.0, r, 0.0, r1, n, st);
    DMRG_CHECK_CUDA(cudaMemcpyAsync(r2, r1, n * 8, cudaMemcpyDeviceToDevice, st));
    DMRG_CHECK_CUDA(cudaMemcpyAsync(y, r1, n * 8, cudaMemcpyDeviceToDevice, st));
    dev_fill(t, 0.0, n, st);
    dev_fill(w, 0.0, n, st);
    dev_fill(w1, 0.0, n, st);
    dev_fill(w2, 0.0, n, st);
    const double beta1 = std::sqrt(std::max(0.0, dot(r1, r1)));
    int it = 0;
    if (beta1 > 0.0) {
        double oldb = 0.0, beta = beta1, dbar = 0.0, epsln = 0.0, phibar = beta1, cs = -1.0, sn = 0.0;
        for (it = 1; it <= max_it; ++it) {
            dev_axpby(1.0 / beta, y, 0.0, v, n, st);
            // y = (I - u u^T)(H - theta) v
            sigma(P, v, y, 1, st);
            dev_axpby(-theta, v, 1.0, y, n, st);
            const double uy = dot(u, y);
            dev_axpby(-uy, u, 1.0, y, n, st);
            if (it >= 2) dev_axpby(-beta / oldb, r1, 1.0, y, n, st);
            const double alfa = dot(v, y);
            dev_axpby(-alfa / beta, r2, 1.0, y, n, st);
            std::swap(r1, r2);
            DMRG_CHECK_CUDA(cudaMemcpyAsync(r2, y, n * 8, cudaMemcpyDeviceToDevice, st));
            oldb = beta;
            beta = std::sqrt(std::max(0.0, dot(r2, r2)));
            const double oldeps = epsln;
            const double delta = cs * dbar + sn * alfa;
            const double gbar = sn * dbar - cs * alfa;
            epsln = sn * beta;
            dbar = -cs * beta;
            const double gamma = std::max(std::sqrt(gbar * gbar + beta * beta), 1e-300);
            cs = gbar / gamma;
            sn = beta / gamma;
            const double phi = cs * phibar;
            phibar = sn * phibar;
            // w = (v - oldeps w1 - delta w2) / gamma with (w1, w2) <- (w2, w)
            std::swap(w1, w2);
            std::swap(w2, w);
            DMRG_CHECK_CUDA(cudaMemcpyAsync(w, v, n * 8, cudaMemcpyDeviceToDevice, st));
            dev_axpby(-oldeps, w1, 1.0, w, n, st);
            dev_axpby(-delta, w2, 1.0, w, n, st);
            dev_axpby(0.0, w, 1.0 / gamma, w, n, st);
            dev_axpby(phi, w, 1.0, t, n, st);
            if (!(phibar == phibar) || phibar <= tol * beta1 || beta <= 1e-300) break;
        }
    }
    P.free(buf, 7 * n);
    return it;
}

}  // namespace

// ---------------------------------------------------------------------------
// Davidson
// ---------------------------------------------------------------------------

namespace {

// Defect-corrected operator around the current vectors X (nr x n,
// orthonormal), with W = H X from the FP64-accurate sigma and P = I - X X^T:
//   H_c = P H_mixed P + W X^T + X W^T - X C X^T,   C = (X^T W + W^T X) / 2.
// H_c X = H X and X^T H_c = X^T H, so every coupling of X in the projected
// Davidson matrix is FP64-accurate (the mixed sigma's own asymmetry would
// otherwise enter there); the mixed error acts only inside the complement of X,
// on the correction, and the Ritz vectors of H_c near X approach H's
// eigenvectors by a factor ~|H - H_mixed| / gap per outer round.
struct DefectCorr {
    int nr = 0;
    const double* X = nullptr;
    const double* W = nullptr;
    double* proj = nullptr;  // nr x n workspace for P v
    std::vector<double> C;
};

struct DavOut {
    std::vector<double> theta, rnorm;
    int iters = 0;
    bool conv = false;
    bool stalled = false;
};

// One Davidson solve from the guesses in psi (nr x n; Ritz vectors on exit).
// stall > 0: stop when the residual no longer falls near the mixed sigma's
// noise floor: after at least kStallMin iterations, the best residual so far
// is below stall * max|theta| and the best of the last kStallWin iterations is
// above 0.7 times the best before them.  (Far above the floor, Davidson may
// stagnate for a while and then converge, so a plateau alone is not a stall.)
// From the next-bond guess of a converged wavefunction the K = 73 residual
// reaches the floor in 4-5 iterations; a window of 3 stops 3 iterations later.
constexpr int kStallMin = 6, kStallWin = 3;
void davidson_run(Plan& P, double* psi, int nr, double tol, int max_iter, int precond, const DefectCorr* corr,
                  double stall, DavOut& out) {
    const int64_t n = P.dim;
    int ms = P.opt.max_space > 0 ? P.opt.max_space : 20 * nr;
    ms = std::max(ms, 3 * nr);
    ms = (int)std::min<int64_t>(ms, n);
    const int64_t need = (int64_t)(2 * ms + 3 * nr + 2) * n + (int64_t)ms * 260 + 3LL * ms * ms + 4 * ms;
    if (need > P.n_dav) {
        P.free(P.d_dav, P.n_dav);
        P.n_dav = need;
        P.d_dav = P.alloc(need);
    }
    double* V = P.d_dav;
    double* W = V + (int64_t)ms * n;
    double* X = W + (int64_t)ms * n;
    double* WY = X + (int64_t)nr * n;
    double* T = WY + (int64_t)nr * n;
    double* hd = T + (int64_t)nr * n;
    double* tmp = hd + n;
    double* dwork = tmp + n;
    double* dco = dwork + (int64_t)ms * 256;
    double* dG = dco + 4 * ms;
    double* dGv = dG + (int64_t)ms * ms;
    double* dev = dGv + (int64_t)ms * ms;
    cudaStream_t st = P.stream;

    // wall time per phase (verbose): diagonal, orthogonalisation, sigma, Ritz
    // step and residuals, preconditioner
    double tph[5] = {0, 0, 0, 0, 0};
    auto tnow = [&]() {
        if (P.opt.verbose) DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
        return std::chrono::steady_clock::now();
    };
    auto tadd = [&](int i, std::chrono::steady_clock::time_point a) {
        if (P.opt.verbose) tph[i] += std::chrono::duration<double, std::milli>(tnow() - a).count();
    };
    // W[0:cnt] = H V[0:cnt] (the defect-corrected operator when one is active)
    std::vector<double> ha((size_t)std::max(nr, 1) * 3);
    auto apply = [&](const double* Vb, double* Wb, int cnt) {
        if (!corr) {
            sigma(P, Vb, Wb, cnt, st);
            return;
        }
        const int q = corr->nr;
        std::vector<std::vector<double>> a(cnt, std::vector<double>(q));
        // P v for every new vector, then one batched mixed sigma
        for (int j = 0; j < cnt; ++j) {
            const double* v = Vb + (int64_t)j * n;
            dev_dots(corr->X, n, q, v, n, dco, dwork, st);
            DMRG_CHECK_CUDA(cudaMemcpyAsync(a[j].data(), dco, q * 8, cudaMemcpyDeviceToHost, st));
            DMRG_CHECK_CUDA(cudaMemcpyAsync(corr->proj + (int64_t)j * n, v, n * 8, cudaMemcpyDeviceToDevice, st));
            dev_combine(corr->X, n, q, dco, n, tmp, st);
            dev_axpby(-1.0, tmp, 1.0, corr->proj + (int64_t)j * n, n, st);
        }
        sigma(P, corr->proj, Wb, cnt, st);
        for (int j = 0; j < cnt; ++j) {
            const double* v = Vb + (int64_t)j * n;
            double* w = Wb + (int64_t)j * n;
            // b = X^T (H_mixed P v), c = W^T v
            dev_dots(corr->X, n, q, w, n, dco, dwork, st);
            dev_dots(corr->W, n, q, v, n, dco + q, dwork, st);
            DMRG_CHECK_CUDA(cudaMemcpyAsync(ha.data(), dco, 2 * q * 8, cudaMemcpyDeviceToHost, st));
            DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
            // H_c v = P (H_mixed P v) + W a + X (c - C a),  a = X^T v
            std::vector<double> cx(q);
            for (int r = 0; r < q; ++r) {
                double s_ = ha[q + r] - ha[r];
                for (int b = 0; b < q; ++b) s_ -= corr->C[(size_t)r * q + b] * a[j][b];
                cx[r] = s_;
            }
            DMRG_CHECK_CUDA(cudaMemcpyAsync(dco, a[j].data(), q * 8, cudaMemcpyHostToDevice, st));
            DMRG_CHECK_CUDA(cudaMemcpyAsync(dco + q, cx.data(), q * 8, cudaMemcpyHostToDevice, st));
            dev_combine(corr->W, n, q, dco, n, tmp, st);
            dev_axpby(1.0, tmp, 1.0, w, n, st);
            dev_combine(corr->X, n, q, dco + q, n, tmp, st);
            dev_axpby(1.0, tmp, 1.0, w, n, st);
            DMRG_CHECK_CUDA(cudaStreamSynchronize(st));  // a[j], cx are host temporaries
        }
    };
    auto tp0 = tnow();
    hdiag(P, hd, st);
    tadd(0, tp0);
    DMRG_CHECK_CUDA(cudaMemcpyAsync(T, psi, (size_t)nr * n * 8, cudaMemcpyDeviceToDevice, st));
    std::vector<double> G((size_t)ms * ms, 0.0);
    std::vector<double> theta(nr, 0.0), rnorm(nr, 0.0);
    std::vector<double> hist;  // largest residual per iteration
    int m = 0, nnew = nr, it = 0;
    bool conv = false, stalled = false;
    EigJob job;
    EigJob* d_job = nullptr;
    DMRG_CHECK_CUDA(cudaMalloc(&d_job, sizeof(EigJob)));
    struct JobFree {
        EigJob*& p;
        ~JobFree() {
            if (p) cudaFree(p);
        }
    } job_free{d_job};
    std::vector<double> Gv;
    std::vector<int> order;
    while (true) {
        // orthonormalise the new directions (classical Gram-Schmidt, twice)
        auto tp1 = tnow();
        int added = 0;
        for (int t = 0; t < nnew; ++t) {
            double* x = T + (int64_t)t * n;
            for (int pass = 0; pass < 2; ++pass) {
                int mm = m + added;
                if (mm == 0) break;
                dev_dots(V, n, mm, x, n, dco, dwork, st);
                dev_combine(V, n, mm, dco, n, tmp, st);
                dev_axpby(-1.0, tmp, 1.0, x, n, st);
            }
            double nrm2 = host_dot(P, x, x, n, dco, dwork);
            if (!(nrm2 == nrm2) || std::isinf(nrm2)) throw Error(DMRG_ENUMERIC, "non-finite Davidson direction");
            double nrm = std::sqrt(nrm2);
            if (nrm > 1e-10) {
                double* dst = V + (int64_t)(m + added) * n;
                dev_axpby(1.0 / nrm, x, 0.0, dst, n, st);
                ++added;
            }
        }
        // fewer independent guesses than roots: add hashed perturbations of the first vector
        for (int tries = 0; m + added < nr && tries < 8 * nr; ++tries) {
            double* x = T;
            if (m + added > 0)
                DMRG_CHECK_CUDA(cudaMemcpyAsync(x, V, n * 8, cudaMemcpyDeviceToDevice, st));
            else
                dev_fill(x, 0.0, n, st);
            dev_perturb(x, n, 7919u + (uint32_t)tries, 1.0, st);
            for (int pass = 0; pass < 2 && m + added > 0; ++pass) {
                dev_dots(V, n, m + added, x, n, dco, dwork, st);
                dev_combine(V, n, m + added, dco, n, tmp, st);
                dev_axpby(-1.0, tmp, 1.0, x, n, st);
            }
            double nrm = std::sqrt(std::max(0.0, host_dot(P, x, x, n, dco, dwork)));
            if (nrm > 1e-10) {
                dev_axpby(1.0 / nrm, x, 0.0, V + (int64_t)(m + added) * n, n, st);
                ++added;
            }
        }
        tadd(1, tp1);
        if (added == 0) break;
        auto tp2 = tnow();
        apply(V + (int64_t)m * n, W + (int64_t)m * n, added);
        tadd(2, tp2);
        auto tp3 = tnow();
        {
            // the new columns of V^T W, read back with one synchronisation
            const int mm = m + added;
            for (int j = m; j < mm; ++j) dev_dots(V, n, mm, W + (int64_t)j * n, n, dGv + (int64_t)(j - m) * mm, dwork, st);
            std::vector<double> cols((size_t)mm * added);
            DMRG_CHECK_CUDA(cudaMemcpyAsync(cols.data(), dGv, cols.size() * 8, cudaMemcpyDeviceToHost, st));
            DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
            for (int j = m; j < mm; ++j)
                for (int i = 0; i < mm; ++i) {
                    const double g = cols[(size_t)(j - m) * mm + i];
                    G[(size_t)i * ms + j] = g;
                    G[(size_t)j * ms + i] = g;
                }
        }
        m += added;
        ++it;
        // Ritz problem on the device (Jacobi)
        std::vector<double> Gs((size_t)m * m);
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) Gs[(size_t)i * m + j] = 0.5 * (G[(size_t)i * ms + j] + G[(size_t)j * ms + i]);
        DMRG_CHECK_CUDA(cudaMemcpyAsync(dG, Gs.data(), (size_t)m * m * 8, cudaMemcpyHostToDevice, st));
        job.A = dG;
        job.V = dGv;
        job.w = dev;
        job.n = m;
        job.lda = m;
        DMRG_CHECK_CUDA(cudaMemcpyAsync(d_job, &job, sizeof(EigJob), cudaMemcpyHostToDevice, st));
        dev_jacobi_eigh_batched(d_job, 1, 40, st);
        std::vector<double> w(m);
        Gv.assign((size_t)m * m, 0.0);
        DMRG_CHECK_CUDA(cudaMemcpyAsync(w.data(), dev, m * 8, cudaMemcpyDeviceToHost, st));
        DMRG_CHECK_CUDA(cudaMemcpyAsync(Gv.data(), dGv, (size_t)m * m * 8, cudaMemcpyDeviceToHost, st));
        DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
        order.resize(m);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return w[a] < w[b]; });
        bool all = true;
        double rmax = 0.0;
        for (int i = 0; i < nr; ++i) {
            int c = order[i];
            theta[i] = w[c];
            std::vector<double> y(m);
            for (int r = 0; r < m; ++r) y[r] = Gv[(size_t)r * m + c];
            DMRG_CHECK_CUDA(cudaMemcpyAsync(dco, y.data(), m * 8, cudaMemcpyHostToDevice, st));
            double* xi = X + (int64_t)i * n;
            double* wy = WY + (int64_t)i * n;
            dev_combine(V, n, m, dco, n, xi, st);
            dev_combine(W, n, m, dco, n, wy, st);
            double* ri = T + (int64_t)i * n;
            DMRG_CHECK_CUDA(cudaMemcpyAsync(ri, wy, n * 8, cudaMemcpyDeviceToDevice, st));
            dev_axpby(-theta[i], xi, 1.0, ri, n, st);
            rnorm[i] = std::sqrt(std::max(0.0, host_dot(P, ri, ri, n, dco + 2 * ms, dwork)));
            if (!(rnorm[i] == rnorm[i])) throw Error(DMRG_ENUMERIC, "non-finite Davidson residual");
            all = all && rnorm[i] <= tol;
            rmax = std::max(rmax, rnorm[i]);
        }
        hist.push_back(rmax);
        tadd(3, tp3);
        if (P.opt.verbose)
            fprintf(stderr, "[dmrg] davidson it=%d m=%d theta0=%.12f |r0|=%.3e\n", it, m, theta[0], rnorm[0]);
        if (all) {
            conv = true;
            break;
        }
        if (it >= max_iter) break;
        if (stall > 0.0 && it >= kStallMin) {
            const double before = *std::min_element(hist.begin(), hist.end() - kStallWin);
            const double recent = *std::min_element(hist.end() - kStallWin, hist.end());
            double tmax = 0.0;
            for (int i = 0; i < nr; ++i) tmax = std::max(tmax, std::fabs(theta[i]));
            if (std::min(before, recent) < stall * tmax && recent > 0.7 * before) {
                stalled = true;
                break;
            }
        }
        // training pairs: the plain method's converged correction for root 0
        if (P.harvest.on) {
            double* tjd = P.alloc(n);
            jd_solve(P, X, theta[0], T, tjd, P.harvest.jd_iters, P.harvest.jd_tol, dco, dwork);
            const double s_ = dev_absmax(hd, theta[0], n, dwork, st);
            const double rmx = dev_absmax(T, 0.0, n, dwork, st);
            P.harvest.pairs += mlp_collect(P.mlp, hd, T, tjd, theta[0], s_, rmx, n, P.harvest.per_solve, st);
            P.free(tjd, n);
        }
        // corrections: diagonal (Jacobi), or scaled per element by the learned g
        auto tp4 = tnow();
        const bool use_mlp = precond == DMRG_PRECOND_MLP && P.mlp.trained && !P.harvest.on;
        if (use_mlp && P.n_mlp_feat < 6 * n) {
            if (P.d_mlp_feat) cudaFree(P.d_mlp_feat);
            P.n_mlp_feat = 6 * n;
            DMRG_CHECK_CUDA(cudaMalloc(&P.d_mlp_feat, P.n_mlp_feat * sizeof(float)));
        }
        for (int i = 0; i < nr; ++i) {
            double* ri = T + (int64_t)i * n;
            if (use_mlp) {
                float* xf = P.d_mlp_feat;
                float* gf = P.d_mlp_feat + 5 * n;
                const double s_ = dev_absmax(hd, theta[i], n, dwork, st);
                const double rmx = dev_absmax(ri, 0.0, n, dwork, st);
                mlp_features(P.mlp, hd, ri, theta[i], s_, rmx, n, xf, st);
                mlp_forward(P.mlp, xf, n, gf, true, st);
                mlp_apply(ri, hd, theta[i], gf, ri, n, st);
            } else {
                dev_jacobi_precond(ri, hd, theta[i], ri, n, st);
            }
        }
        if (precond == DMRG_PRECOND_MLP && !use_mlp) P.stats.precond_fallbacks += nr;
        tadd(4, tp4);
        nnew = nr;
        if (m + nr > ms) {  // restart with the Ritz vectors
            DMRG_CHECK_CUDA(cudaMemcpyAsync(V, X, (size_t)nr * n * 8, cudaMemcpyDeviceToDevice, st));
            DMRG_CHECK_CUDA(cudaMemcpyAsync(W, WY, (size_t)nr * n * 8, cudaMemcpyDeviceToDevice, st));
            std::fill(G.begin(), G.end(), 0.0);
            for (int i = 0; i < nr; ++i) G[(size_t)i * ms + i] = theta[i];
            m = nr;
        }
    }
    if (P.opt.verbose)
        fprintf(stderr, "[dmrg] davidson phases (ms): diagonal %.0f, orthogonalisation %.0f, sigma %.0f, "
                        "Ritz+residual %.0f, preconditioner %.0f\n",
                tph[0], tph[1], tph[2], tph[3], tph[4]);
    DMRG_CHECK_CUDA(cudaMemcpyAsync(psi, X, (size_t)nr * n * 8, cudaMemcpyDeviceToDevice, st));
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    out.theta = theta;
    out.rnorm = rnorm;
    out.iters = it;
    out.conv = conv;
    out.stalled = stalled;
}

// FP64-accurate Rayleigh quotients and residual norms of the nr vectors X
// (orthonormal); Wacc receives H X.
void accurate_residuals(Plan& P, const double* X, int nr, double* Wacc, double* r, std::vector<double>& theta,
                        std::vector<double>& rnorm, double* dco, double* dwork) {
    const int64_t n = P.dim;
    cudaStream_t st = P.stream;
    sigma_fp64(P, X, Wacc, nr, st);
    theta.assign(nr, 0.0);
    rnorm.assign(nr, 0.0);
    for (int i = 0; i < nr; ++i) {
        const double* xi = X + (int64_t)i * n;
        const double* wi = Wacc + (int64_t)i * n;
        const double num = host_dot(P, xi, wi, n, dco, dwork);
        const double den = host_dot(P, xi, xi, n, dco, dwork);
        theta[i] = num / den;
        DMRG_CHECK_CUDA(cudaMemcpyAsync(r, wi, n * 8, cudaMemcpyDeviceToDevice, st));
        dev_axpby(-theta[i], xi, 1.0, r, n, st);
        rnorm[i] = std::sqrt(std::max(0.0, host_dot(P, r, r, n, dco, dwork)));
        if (!(rnorm[i] == rnorm[i])) throw Error(DMRG_ENUMERIC, "non-finite FP64 residual");
    }
}

}  // namespace

dmrg_status davidson(Plan& P, double* psi, int nr, double tol, int max_iter, int precond,
                     double* energies, int* iters) {
    DMRG_REQUIRE(P.bond > 0, DMRG_EINVAL, "no current bond");
    DMRG_REQUIRE(nr >= 1 && nr <= 16, DMRG_EINVAL, "n_roots must be in 1..16");
    const int64_t n = P.dim;
    DMRG_REQUIRE(n >= nr, DMRG_EINVAL, "fewer states than roots at this bond");
    cudaStream_t st = P.stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    const bool refine = P.mixed() && P.opt.refine && !P.harvest.on;
    DavOut o;
    int rounds = 0, total_it = 0;
    double rmax = 0.0;
    bool conv = false;
    // the mixed iteration stops at its noise floor instead of running to max_iter;
    // the floor of the sigma relative to |theta| is ~1e-5 with two or three bf16
    // pieces and ~3e-3 with one (measured), so a plateau counts as a stall only
    // within ~10x of it
    const double stall = !P.mixed() ? 0.0 : (P.nsplit == 1 ? 3e-2 : 1e-4);
    davidson_run(P, psi, nr, tol, max_iter, precond, nullptr, stall, o);
    total_it += o.iters;
    std::vector<double> theta = o.theta;
    if (refine) {
        const int max_rounds = P.opt.max_refine > 0 ? P.opt.max_refine : 8;
        // X copy, H X (accurate), projection workspace, residual, small buffers
        const int64_t nbuf = 3 * (int64_t)nr * n + n + 512;
        double* buf = P.alloc(nbuf);
        double* Xc = buf;
        double* Wacc = Xc + (int64_t)nr * n;
        double* proj = Wacc + (int64_t)nr * n;
        double* r = proj + (int64_t)nr * n;
        double* dco = r + n;
        double* dwork = dco + 64;
        std::vector<double> rn;
        try {
            for (;;) {
                accurate_residuals(P, psi, nr, Wacc, r, theta, rn, dco, dwork);
                rmax = *std::max_element(rn.begin(), rn.end());
                if (P.opt.verbose)
                    fprintf(stderr, "[dmrg] refine round %d: FP64 theta0=%.12f |r|max=%.3e (inner its %d%s)\n", rounds,
                            theta[0], rmax, o.iters, o.stalled ? ", stalled" : "");
                if (rmax <= tol) {
                    conv = true;
                    break;
                }
                if (rounds >= max_rounds) break;
                // the corrected operator around X: C = sym(X^T W)
                DefectCorr corr;
                corr.nr = nr;
                DMRG_CHECK_CUDA(cudaMemcpyAsync(Xc, psi, (size_t)nr * n * 8, cudaMemcpyDeviceToDevice, st));
                corr.X = Xc;  // psi receives the new Ritz vectors
                corr.W = Wacc;
                corr.proj = proj;
                corr.C.assign((size_t)nr * nr, 0.0);
                std::vector<double> xw((size_t)nr * nr);
                for (int a = 0; a < nr; ++a)
                    for (int b = 0; b < nr; ++b)
                        xw[(size_t)a * nr + b] = host_dot(P, Xc + (int64_t)a * n, Wacc + (int64_t)b * n, n, dco, dwork);
                for (int a = 0; a < nr; ++a)
                    for (int b = 0; b < nr; ++b) corr.C[(size_t)a * nr + b] = 0.5 * (xw[(size_t)a * nr + b] + xw[(size_t)b * nr + a]);
                const double tol_in = std::max(0.5 * tol, 0.1 * rmax);
                // no floor to stall at: H_c reproduces H on X, and its mixed error acts
                // on the small correction only
                davidson_run(P, psi, nr, tol_in, max_iter, precond, &corr, 0.0, o);
                total_it += o.iters;
                ++rounds;
            }
        } catch (...) {
            P.free(buf, nbuf);
            throw;
        }
        P.free(buf, nbuf);
    } else {
        conv = o.conv;
        rmax = o.rnorm.empty() ? 0.0 : *std::max_element(o.rnorm.begin(), o.rnorm.end());
        if (P.mixed() && P.opt.fp64_final) {
            // FP64 Rayleigh quotients <x|H|x> of the mixed-precision Ritz vectors
            double* buf = P.alloc(2 * n + 512);
            std::vector<double> rn;
            try {
                for (int i = 0; i < nr; ++i) {
                    std::vector<double> th1;
                    accurate_residuals(P, psi + (int64_t)i * n, 1, buf, buf + n, th1, rn, buf + 2 * n, buf + 2 * n + 64);
                    theta[i] = th1[0];
                }
            } catch (...) {
                P.free(buf, 2 * n + 512);
                throw;
            }
            P.free(buf, 2 * n + 512);
        }
    }
    cudaEventRecord(e1, st);
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    float ms_ = 0.f;
    cudaEventElapsedTime(&ms_, e0, e1);
    P.stats.ms_davidson += ms_;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int i = 0; i < nr; ++i) energies[i] = theta[i] + P.I.e_core;
    if (iters) *iters = total_it;
    P.stats.davidson_iters_last = total_it;
    P.stats.davidson_rnorm_last = rmax;
    P.stats.davidson_conv_last = conv ? 1 : 0;
    P.stats.davidson_stalled_last = o.stalled ? 1 : 0;
    P.stats.davidson_refine_last = rounds;
    return conv ? DMRG_OK : DMRG_ENOTCONV;
}

// ---------------------------------------------------------------------------
// Decimation
// ---------------------------------------------------------------------------

namespace {
struct Comp {
    int a, b;  // forward: (il, c1) ; backward: (c2, ir)
    int dim;
    int64_t off;
};
struct Group {
    QN q;
    std::vector<Comp> rows;
    std::map<std::pair<int, int>, int> rindex;
    int n = 0;
    int64_t rho_off = 0;
    std::vector<double> w;
    std::vector<int> kept;  // column indices of V_q
};
}  // namespace

void decimate(Plan& P, const double* psi, int nr, int Dmax, bool forward, double* discarded) {
    DMRG_REQUIRE(P.bond > 0, DMRG_EINVAL, "no current bond");
    const int k = P.bond, K = P.K;
    DMRG_REQUIRE(forward ? (k + 1 <= K - 1) : (k - 1 >= 1), DMRG_EINVAL, "cannot move past the chain end");
    cudaStream_t st = P.stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    const auto bl = P.mps.bonds[k - 1];
    const auto br = P.mps.bonds[k + 1];
    // the bond's intermediates are not needed any more (the next bond forms its
    // own); freeing them first lowers the peak of the renormalisation below
    free_interms(P, P.interm);
    P.bond = -1;  // no sigma at this bond any more (its intermediates are gone)
    // groups by the label of bond k
    std::map<QN, Group> groups;
    for (const Plan::Sector& s : P.layout) {
        int c1 = s.y / 4, c2 = s.y % 4;
        QN q = QN(bl[s.il][0], bl[s.il][1]) + kSiteQN[c1];
        Group& g = groups[q];
        g.q = q;
        std::pair<int, int> key = forward ? std::make_pair(s.il, c1) : std::make_pair(c2, s.ir);
        if (!g.rindex.count(key)) {
            g.rindex[key] = (int)g.rows.size();
            g.rows.push_back({key.first, key.second, forward ? s.dl : s.dr, (int64_t)g.n});
            g.n += forward ? s.dl : s.dr;
        }
    }
    int64_t rho_tot = 0;
    for (auto& kv : groups) {
        kv.second.rho_off = rho_tot;
        rho_tot += (int64_t)kv.second.n * kv.second.n;
    }
    double* d_rho = P.alloc(2 * rho_tot + rho_tot / 1 + 64);
    double* d_vec = d_rho + rho_tot;
    double* d_w = d_vec + rho_tot;
    // rho_q = (1/nr) sum_roots M M^T (forward) or M^T M (backward)
    WorkList wl;
    P.f64_tiles(wl);
    for (auto& kv : groups) {
        Group& g = kv.second;
        std::map<std::pair<int, int>, std::vector<Seg>> blk;  // (row comp, col comp) -> segs
        // list sectors of this group
        std::vector<const Plan::Sector*> secs;
        for (const Plan::Sector& s : P.layout) {
            QN q = QN(bl[s.il][0], bl[s.il][1]) + kSiteQN[s.y / 4];
            if (q == g.q) secs.push_back(&s);
        }
        for (const Plan::Sector* a : secs)
            for (const Plan::Sector* b : secs) {
                int ra, rb;
                Seg sg{};
                if (forward) {
                    if (a->y % 4 != b->y % 4 || a->ir != b->ir) continue;  // same column comp (c2, ir)
                    ra = g.rindex[{a->il, a->y / 4}];
                    rb = g.rindex[{b->il, b->y / 4}];
                    sg.a_off = a->off;
                    sg.lda = a->dr;
                    sg.a_tr = 0;
                    sg.b_off = b->off;
                    sg.ldb = b->dr;
                    sg.b_tr = 1;
                    sg.k = a->dr;
                } else {
                    if (a->il != b->il || a->y / 4 != b->y / 4) continue;  // same column comp (il, c1)
                    ra = g.rindex[{a->y % 4, a->ir}];
                    rb = g.rindex[{b->y % 4, b->ir}];
                    sg.a_off = a->off;
                    sg.lda = a->dr;
                    sg.a_tr = 1;
                    sg.b_off = b->off;
                    sg.ldb = b->dr;
                    sg.b_tr = 0;
                    sg.k = a->dl;
                }
                sg.a_buf = BUF_PSI;
                sg.b_buf = BUF_PSI;
                sg.alpha = 1.0 / nr;
                for (int v = 0; v < nr; ++v) {
                    Seg s2 = sg;
                    s2.a_off += (int64_t)v * P.dim;
                    s2.b_off += (int64_t)v * P.dim;
                    blk[{ra, rb}].push_back(s2);
                }
            }
        for (auto& bk : blk) {
            const Comp& ca = g.rows[bk.first.first];
            const Comp& cb = g.rows[bk.first.second];
            wl.add_block(g.rho_off + ca.off * g.n + cb.off, BUF_OUT, ca.dim, cb.dim, g.n, bk.second, TILE_STORE);
        }
    }
    DMRG_CHECK_CUDA(cudaMemsetAsync(d_rho, 0, rho_tot * 8, st));
    wl.upload(st);
    BufTable bt{};
    bt.p[BUF_PSI] = const_cast<double*>(psi);
    bt.p[BUF_OUT] = d_rho;
    const auto hd0 = std::chrono::steady_clock::now();
    launch_seg_gemm_f64(wl, bt, 1, st);
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    const auto hd1 = std::chrono::steady_clock::now();
    // eigen-decomposition of every rho_q
    std::vector<EigJob> jobs;
    int64_t woff = 0;
    for (auto& kv : groups) {
        Group& g = kv.second;
        EigJob j;
        j.A = d_rho + g.rho_off;
        j.V = d_vec + g.rho_off;
        j.w = d_w + woff;
        j.n = g.n;
        j.lda = g.n;
        woff += g.n;
        jobs.push_back(j);
        DMRG_REQUIRE(g.n <= 16384, DMRG_EINVAL, "density-matrix sector larger than 16384");
    }
    std::vector<double> conv;
    P.stats.decim_sweeps_last = block_jacobi_eigh(
        jobs, 40, 1e-14, st, [&](int64_t n) { return P.alloc(n); }, [&](double* p, int64_t n) { P.free(p, n); },
        &conv, &P.stats.decim_sweeps32_last, P.opt.decim_tol32, P.opt.decim_fp64_units == 0);
    for (int i = 0; i < 41; ++i) P.stats.decim_conv_last[i] = i < (int)conv.size() ? conv[i] : 0.0;
    P.stats.decim_nmat_last = (int)jobs.size();
    P.stats.decim_nmax_last = 0;
    for (auto& j : jobs) P.stats.decim_nmax_last = std::max(P.stats.decim_nmax_last, (int)j.n);
    const auto hd2 = std::chrono::steady_clock::now();
    std::vector<double> hw(woff), hv(rho_tot);
    DMRG_CHECK_CUDA(cudaMemcpyAsync(hw.data(), d_w, woff * 8, cudaMemcpyDeviceToHost, st));
    DMRG_CHECK_CUDA(cudaMemcpyAsync(hv.data(), d_vec, rho_tot * 8, cudaMemcpyDeviceToHost, st));
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    wl.release();
    P.free(d_rho, 2 * rho_tot + rho_tot + 64);
    // choose the kept states: largest weights, ties by group order then rank
    struct Cand {
        double w;
        int g, rank, col;
    };
    std::vector<Cand> cands;
    std::vector<Group*> glist;
    woff = 0;
    for (auto& kv : groups) {
        Group& g = kv.second;
        g.w.assign(hw.begin() + woff, hw.begin() + woff + g.n);
        woff += g.n;
        std::vector<int> ord(g.n);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return g.w[a] > g.w[b]; });
        for (int r = 0; r < g.n; ++r) cands.push_back({g.w[ord[r]], (int)glist.size(), r, ord[r]});
        glist.push_back(&g);
    }
    std::stable_sort(cands.begin(), cands.end(), [](const Cand& a, const Cand& b) {
        if (a.w != b.w) return a.w > b.w;
        if (a.g != b.g) return a.g < b.g;
        return a.rank < b.rank;
    });
    double wdisc = 0.0;
    int nkept = 0;
    for (const Cand& c : cands) {
        if (nkept < Dmax && c.w > 1e-28) {
            glist[c.g]->kept.push_back(c.col);
            ++nkept;
        } else {
            wdisc += std::max(c.w, 0.0);
        }
    }
    if (discarded) *discarded = wdisc;
    // new bond-k sectors (group order) and the new site tensor
    std::vector<std::array<int, 3>> newbond;
    std::map<std::array<int, 3>, std::vector<double>> newsite;
    std::map<QN, int> newidx;
    for (auto& kv : groups) {
        Group& g = kv.second;
        if (g.kept.empty()) continue;
        // keep columns in descending-weight order (rank order)
        std::stable_sort(g.kept.begin(), g.kept.end(), [&](int a, int b) { return g.w[a] > g.w[b]; });
        newidx[g.q] = (int)newbond.size();
        newbond.push_back({g.q.n, g.q.s, (int)g.kept.size()});
    }
    for (auto& kv : groups) {
        Group& g = kv.second;
        if (g.kept.empty()) continue;
        const int inew = newidx[g.q];
        const int nk = (int)g.kept.size();
        const double* Vq = hv.data() + g.rho_off;
        for (const Comp& c : g.rows) {
            std::vector<double> blk((size_t)c.dim * nk);
            for (int a = 0; a < c.dim; ++a)
                for (int t = 0; t < nk; ++t) blk[(size_t)a * nk + t] = Vq[(size_t)(c.off + a) * g.n + g.kept[t]];
            if (forward) {
                newsite[{c.a, c.b, inew}] = std::move(blk);  // (il, c1, new): d_il x nk
            } else {
                std::vector<double> bt_((size_t)nk * c.dim);  // (new, c2, ir): nk x d_ir
                for (int a = 0; a < c.dim; ++a)
                    for (int t = 0; t < nk; ++t) bt_[(size_t)t * c.dim + a] = blk[(size_t)a * nk + t];
                newsite[{inew, c.a, c.b}] = std::move(bt_);
            }
        }
    }
    // install into the MPS and drop stale environments
    std::vector<Plan::Sector> old_layout = P.layout;
    const int64_t old_dim = P.dim;
    P.mps.bonds[k] = newbond;
    if (forward) {
        P.mps.sites[k] = newsite;
        P.mps.center = k + 1;
        for (int m = k; m <= K; ++m)
            free_block(P, P.left[m]);
        for (int m = 0; m <= k - 1; ++m)
            free_block(P, P.right[m]);
    } else {
        P.mps.sites[k + 1] = newsite;
        P.mps.center = k - 1;
        for (int m = 0; m <= k; ++m)
            free_block(P, P.right[m]);
        for (int m = k + 1; m <= K; ++m)
            free_block(P, P.left[m]);
    }
    const auto hd3 = std::chrono::steady_clock::now();
    // guess for the next bond: U^T Psi A[k+2] (forward) or A[k-1] Psi V (backward)
    const int kn = forward ? k + 1 : k - 1;
    const auto nbl = P.mps.bonds[kn - 1];
    const auto nbr = P.mps.bonds[kn + 1];
    std::map<std::pair<int, int>, int> ridx;
    for (int i = 0; i < (int)nbr.size(); ++i) ridx[{nbr[i][0], nbr[i][1]}] = i;
    struct NSec {
        int il, y, ir;
        int64_t off;
        int dl, dr;
    };
    std::vector<NSec> nl;
    std::map<std::pair<int, int>, int> nsec_of;
    int64_t ndim = 0;
    for (int il = 0; il < (int)nbl.size(); ++il)
        for (int y = 0; y < 16; ++y) {
            QN q = QN(nbl[il][0], nbl[il][1]) + kSiteQN[y / 4] + kSiteQN[y % 4];
            auto it = ridx.find({q.n, q.s});
            if (it == ridx.end()) continue;
            nsec_of[{il, y}] = (int)nl.size();
            nl.push_back({il, y, it->second, ndim, nbl[il][2], nbr[it->second][2]});
            ndim += (int64_t)nbl[il][2] * nbr[it->second][2];
        }
    P.free(P.d_guess, P.n_guess);
    P.n_guess = std::max<int64_t>((int64_t)nr * ndim, 1);
    P.d_guess = P.alloc(P.n_guess);
    P.guess_nr = nr;
    double* next_psi = P.d_guess;
    {
        // device copies of the two site tensors used
        const int sa = forward ? k : k - 1;       // U (new A[k]) or A[k-1]
        const int sb = forward ? k + 2 : k + 1;   // A[k+2] or V (new A[k+1])
        auto upload = [&](int site, std::map<std::array<int, 3>, int64_t>& off, int64_t& nn) {
            int64_t tot = 0;
            for (auto& kv : P.mps.sites[site]) {
                off[kv.first] = tot;
                tot += (int64_t)kv.second.size();
            }
            nn = std::max<int64_t>(tot, 1);
            double* d = P.alloc(nn);
            std::vector<double> h(nn, 0.0);
            for (auto& kv : P.mps.sites[site]) std::copy(kv.second.begin(), kv.second.end(), h.begin() + off[kv.first]);
            DMRG_CHECK_CUDA(cudaMemcpyAsync(d, h.data(), nn * 8, cudaMemcpyHostToDevice, st));
            DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
            return d;
        };
        std::map<std::array<int, 3>, int64_t> offa, offb;
        int64_t na = 0, nb = 0;
        double* da = upload(sa, offa, na);
        double* db = upload(sb, offb, nb);
        ProductList pl;
        for (auto& s : nl) pl.outs.push_back({BUF_OUT, s.off, s.dl, s.dr, s.dr});
        for (const Plan::Sector& s : old_layout) {
            const int c1 = s.y / 4, c2 = s.y % 4;
            if (forward) {
                // old (il, c1, c2, ir) with U(il, c1, new) and A[k+2](ir, c3, ir')
                QN q = QN(bl[s.il][0], bl[s.il][1]) + kSiteQN[c1];
                auto ni = newidx.find(q);
                if (ni == newidx.end()) continue;
                auto ua = offa.find({s.il, c1, ni->second});
                if (ua == offa.end()) continue;
                const int nk = newbond[ni->second][2];
                for (int c3 = 0; c3 < 4; ++c3) {
                    for (auto& kv : P.mps.sites[sb]) {
                        if (kv.first[0] != s.ir || kv.first[1] != c3) continue;
                        const int ir2 = kv.first[2];
                        auto os = nsec_of.find({ni->second, c2 * 4 + c3});
                        if (os == nsec_of.end()) continue;
                        const NSec& o = nl[os->second];
                        if (o.ir != ir2) continue;
                        Contrib c;
                        c.out = os->second;
                        c.P.buf = BUF_L;
                        c.P.off = ua->second;
                        c.P.ld = nk;
                        c.P.tr = true;   // U^T : nk x d_il
                        c.Q.buf = BUF_PSI;
                        c.Q.off = s.off;
                        c.Q.ld = s.dr;   // Psi : d_il x d_ir
                        c.R.buf = BUF_R;
                        c.R.off = offb[kv.first];
                        c.R.ld = o.dr;   // A[k+2](ir, c3, ir2) : d_ir x d_ir2
                        c.m = nk;
                        c.k1 = s.dl;
                        c.k2 = s.dr;
                        c.n = o.dr;
                        c.alpha = 1.0;
                        pl.cs.push_back(c);
                    }
                }
            } else {
                // old (il, c1, c2, ir) with A[k-1](il0, c0, il) and V(new, c2, ir)
                QN q = QN(br[s.ir][0], br[s.ir][1]) - kSiteQN[c2];
                auto ni = newidx.find(q);
                if (ni == newidx.end()) continue;
                auto vb = offb.find({ni->second, c2, s.ir});
                if (vb == offb.end()) continue;
                const int nk = newbond[ni->second][2];
                for (auto& kv : P.mps.sites[sa]) {
                    if (kv.first[2] != s.il) continue;
                    const int il0 = kv.first[0], c0 = kv.first[1];
                    auto os = nsec_of.find({il0, c0 * 4 + c1});
                    if (os == nsec_of.end()) continue;
                    const NSec& o = nl[os->second];
                    if (o.ir != ni->second) continue;
                    Contrib c;
                    c.out = os->second;
                    c.P.buf = BUF_L;
                    c.P.off = offa[kv.first];
                    c.P.ld = s.dl;    // A[k-1](il0, c0, il) : d_il0 x d_il
                    c.Q.buf = BUF_PSI;
                    c.Q.off = s.off;
                    c.Q.ld = s.dr;    // Psi : d_il x d_ir
                    c.R.buf = BUF_R;
                    c.R.off = vb->second;
                    c.R.ld = s.dr;
                    c.R.tr = true;    // V^T : d_ir x nk
                    c.m = o.dl;
                    c.k1 = s.dl;
                    c.k2 = s.dr;
                    c.n = nk;
                    c.alpha = 1.0;
                    pl.cs.push_back(c);
                }
            }
        }
        int maxd = 1;
        for (auto& b : nbl) maxd = std::max(maxd, b[2]);
        for (auto& b : nbr) maxd = std::max(maxd, b[2]);
        for (auto& b : bl) maxd = std::max(maxd, b[2]);
        for (auto& b : br) maxd = std::max(maxd, b[2]);
        ensure_ident(P, maxd);
        P.f64_tiles(pl);
        pl.lower(BUF_SCR, BUF_ID, P.ident_n, scratch_cap_f64(P), 1 << 14);
        ensure_scratch_f64(P, std::max<int64_t>(pl.scratch_elems, 1) * nr);
        pl.upload(st);
        DMRG_CHECK_CUDA(cudaMemsetAsync(next_psi, 0, (size_t)nr * ndim * 8, st));
        BufTable b2{};
        b2.p[BUF_L] = da;
        b2.p[BUF_R] = db;
        b2.p[BUF_PSI] = const_cast<double*>(psi);
        b2.p[BUF_SCR] = P.d_scratch;
        b2.p[BUF_ID] = P.d_ident;
        b2.p[BUF_OUT] = next_psi;
        b2.vstride[BUF_PSI] = old_dim;
        b2.vstride[BUF_OUT] = ndim;
        b2.vstride[BUF_SCR] = std::max<int64_t>(pl.scratch_elems, 1);
        pl.run(b2, nr, st);
        DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
        pl.release();
        P.free(da, na);
        P.free(db, nb);
    }
    P.bond = -1;
    cudaEventRecord(e1, st);
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    const auto hd4 = std::chrono::steady_clock::now();
    auto span = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
        return std::chrono::duration<double, std::milli>(b - a).count();
    };
    P.stats.ms_decim_parts[0] += span(hd0, hd1);  // density matrices
    P.stats.ms_decim_parts[1] += span(hd1, hd2);  // eigensolver
    P.stats.ms_decim_parts[2] += span(hd2, hd3);  // selection and new site tensor (host)
    P.stats.ms_decim_parts[3] += span(hd3, hd4);  // next-bond guess
    float ms_ = 0.f;
    cudaEventElapsedTime(&ms_, e0, e1);
    P.stats.ms_decim += ms_;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    set_bond(P, kn);  // renormalises the grown block and plans the next bond
}

// Two-site tensor A[k] A[k+1] of the current MPS, in the canonical layout.
void two_site_guess(Plan& P, double* out) {
    const int k = P.bond;
    cudaStream_t st = P.stream;
    const auto& bm = P.mps.bonds[k];
    std::map<std::array<int, 3>, int64_t> offa, offb;
    int64_t na = 0, nb = 0;
    auto upload = [&](int site, std::map<std::array<int, 3>, int64_t>& off, int64_t& nn) {
        int64_t tot = 0;
        for (auto& kv : P.mps.sites[site]) {
            off[kv.first] = tot;
            tot += (int64_t)kv.second.size();
        }
        nn = std::max<int64_t>(tot, 1);
        double* d = P.alloc(nn);
        std::vector<double> h(nn, 0.0);
        for (auto& kv : P.mps.sites[site]) std::copy(kv.second.begin(), kv.second.end(), h.begin() + off[kv.first]);
        DMRG_CHECK_CUDA(cudaMemcpyAsync(d, h.data(), nn * 8, cudaMemcpyHostToDevice, st));
        DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
        return d;
    };
    double* da = upload(k, offa, na);
    double* db = upload(k + 1, offb, nb);
    WorkList wl;
    P.f64_tiles(wl);
    for (const Plan::Sector& s : P.layout) {
        const int c1 = s.y / 4, c2 = s.y % 4;
        std::vector<Seg> segs;
        for (int im = 0; im < (int)bm.size(); ++im) {
            auto a = offa.find({s.il, c1, im});
            auto b = offb.find({im, c2, s.ir});
            if (a == offa.end() || b == offb.end()) continue;
            Seg sg{};
            sg.a_off = a->second;
            sg.lda = bm[im][2];
            sg.b_off = b->second;
            sg.ldb = s.dr;
            sg.k = bm[im][2];
            sg.a_buf = BUF_L;
            sg.b_buf = BUF_R;
            sg.alpha = 1.0;
            segs.push_back(sg);
        }
        wl.add_block(s.off, BUF_OUT, s.dl, s.dr, s.dr, segs, TILE_STORE);
    }
    wl.upload(st);
    BufTable bt{};
    bt.p[BUF_L] = da;
    bt.p[BUF_R] = db;
    bt.p[BUF_OUT] = out;
    launch_seg_gemm_f64(wl, bt, 1, st);
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    wl.release();
    P.free(da, na);
    P.free(db, nb);
}

// ---------------------------------------------------------------------------
// Sweep
// ---------------------------------------------------------------------------

dmrg_status sweep(Plan& P, int n_sweeps, const int* D_schedule, double* energies, double* discarded) {
    DMRG_REQUIRE(P.mps.center == 1, DMRG_EINVAL, "sweeps start from an MPS centred on bond (1,2)");
    const int K = P.K;
    const int nr = P.opt.n_roots;
    const int keep = P.opt.keep_envs;
    P.opt.keep_envs = 1;
    if (P.bond != 1) set_bond(P, 1);
    int64_t psi_n = (int64_t)nr * P.dim;
    double* psi = P.alloc(psi_n);
    two_site_guess(P, psi);
    for (int v = 1; v < nr; ++v) {
        DMRG_CHECK_CUDA(cudaMemcpyAsync(psi + (int64_t)v * P.dim, psi, P.dim * 8, cudaMemcpyDeviceToDevice, P.stream));
        dev_perturb(psi + (int64_t)v * P.dim, P.dim, 1000u + v, 0.5, P.stream);
    }
    dmrg_status last = DMRG_OK;
    std::vector<double> en(nr);
    for (int sw = 0; sw < n_sweeps; ++sw) {
        const int D = D_schedule ? D_schedule[sw] : P.D;
        double wmax = 0.0;
        std::vector<std::pair<int, bool>> steps;
        for (int k = 1; k <= K - 2; ++k) steps.push_back({k, true});
        for (int k = K - 1; k >= 2; --k) steps.push_back({k, false});
        for (auto& step : steps) {
            const int k = step.first;
            if (P.bond != k) set_bond(P, k);
            tier_policy(P, k, step.second);  // copies overlap this bond's Davidson
            int iters = 0;
            dmrg_status s = davidson(P, psi, nr, P.opt.tol, P.opt.max_iter, P.opt.precond, en.data(), &iters);
            if (s == DMRG_ENOTCONV) last = s;
            if (P.opt.verbose)
                fprintf(stderr, "[dmrg] sweep %d bond %d %s E=%.12f iters=%d\n", sw, k, step.second ? "fwd" : "bwd",
                        en[0], iters);
            double w = 0.0;
            decimate(P, psi, nr, D, step.second, &w);
            wmax = std::max(wmax, w);
            P.free(psi, psi_n);
            psi = P.d_guess;
            psi_n = P.n_guess;
            P.d_guess = nullptr;
            P.n_guess = 0;
        }
        energies[sw] = en[0];
        if (discarded) discarded[sw] = wmax;
    }
    P.free(psi, psi_n);
    P.opt.keep_envs = keep;
    return last;
}

}  // namespace dmrg

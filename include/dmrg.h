/*
 * dmrg.h -- C-ABI of libdmrg.so: the two-site ab initio DMRG hot path
 * (arXiv:2311.02854) on one GB300 (sm_103a).
 *
 * The library computes the Davidson sigma product sigma = H psi of Eq. (Sigma)
 * for the two-site wavefunction of Sec. 2.1, with the renormalised normal and
 * complementary operators of Eq. (qops) kept in device memory, the
 * renormalisation update of Eq. (Renorm), the Davidson eigensolver and the
 * decimation step (Sec. 2.1, 2.3).  Every arithmetic step runs in the
 * library's own CUDA kernels; the host only plans (index tables, integral
 * coefficient tables, the choice of kept states from eigenvalues).
 *
 * Conventions
 *  - Spin orbital p = 2*i + s (s = 0 alpha, 1 beta) of spatial orbital i;
 *    Jordan-Wigner order (1a, 1b, 2a, 2b, ...).
 *  - Local basis of a site (Sec. 2.1, after Eq. MPS): n = 0 vac, 1 beta,
 *    2 alpha, 3 alpha-beta, with |ab> = a+_a a+_b |vac>.
 *  - Hamiltonian Eq. (Hsq) with h (K x K) and chemist integrals
 *    (pq|rs) = sum_X chol[X][p][q] chol[X][r][s].
 *  - Two-site wavefunction layout ("canonical layout"): sectors ordered by
 *    (left sector il, c1 = 0..3, c2 = 0..3), the right sector being the one
 *    whose bond label is label(il) + q(c1) + q(c2); each sector block is
 *    d_l x d_r, row-major, blocks packed back to back (see dmrg_layout).
 *  - Bond b lies between sites b and b+1 (sites numbered 1..K); bond labels
 *    are the (N, 2Sz) quantum numbers of sites 1..b.
 *
 * Ownership: psi / sigma / diag buffers are owned by the caller.  A plan owns
 * every device allocation it makes (operator store, intermediates, work
 * lists, scratch) and frees it in dmrg_destroy.
 *
 * Errors: every call returns a dmrg_status; nothing aborts.  A device-side
 * failure (a kernel wait that gave up, a NaN seen by a check) is reported
 * through a device error word read after the stream synchronises.
 * dmrg_last_error() gives a one-line description of the last failure.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls are synchronous with respect to the host unless stated.
 */
#ifndef DMRG_H
#define DMRG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmrg_plan_s* dmrg_plan_t;

typedef enum {
    DMRG_OK = 0,
    DMRG_EINVAL = -1,     /* bad argument (sizes, quantum numbers, file) */
    DMRG_ENOMEM = -2,     /* device allocation would exceed the budget / failed */
    DMRG_ECUDA = -3,      /* a CUDA runtime call failed */
    DMRG_ENUMERIC = -4,   /* NaN/Inf or breakdown detected */
    DMRG_ETIMEOUT = -5,   /* a bounded device wait gave up */
    DMRG_ENOTCONV = -6,   /* Davidson did not reach the tolerance */
    DMRG_EIO = -7         /* file could not be read or written */
} dmrg_status;

/* Arithmetic of the operator store and of the sigma / renormalisation GEMMs.
 * FP64: everything in double precision (reference GPU path).
 * BF16X3: operators, wavefunction and intermediates split x = hi + lo into two
 *   bf16 numbers; each product uses hi*hi + hi*lo + lo*hi on the tcgen05
 *   tensor cores with FP32 accumulation in tensor memory; sigma is summed
 *   into FP64.  Davidson, orthogonalisation, Ritz, residuals, energies and
 *   decimation stay FP64.
 * BF16: as BF16X3 with only the hi part (one product per tile).
 * BF16X6: three pieces x = hi + lo + lo2 (24 significant bits, FP32-like
 *   storage) and the six products whose piece orders sum to at most 2.
 * FP64_TC: FP64 operator store and results, every product FP64-accurate on the
 *   bf16 tensor cores (error-free splitting, Ozaki et al. 2012: per 32-deep K
 *   stage each row of A and column of B is scaled by a power of two and cut
 *   into six 8-bit slices; the slice products whose orders sum to <= 5
 *   accumulate exactly in FP32 tensor memory, one accumulator per order;
 *   the orders are combined in double-float arithmetic and written as FP64).
 *   Per product, the error is bounded by about 2^-45 times the row and column
 *   maxima times the depth; not bitwise FP64, no FP64 arithmetic units. */
typedef enum { DMRG_FP64 = 0, DMRG_BF16X3 = 1, DMRG_BF16 = 2, DMRG_BF16X6 = 3, DMRG_FP64_TC = 4 } dmrg_precision;

typedef enum { DMRG_PRECOND_JACOBI = 0, DMRG_PRECOND_MLP = 1 } dmrg_precond;

typedef struct {
    int precision;          /* dmrg_precision */
    int n_roots;            /* roots kept by Davidson (state-averaged decimation if > 1) */
    double tol;             /* Davidson residual 2-norm tolerance */
    int max_iter;           /* Davidson iterations per bond */
    int max_space;          /* Davidson subspace size (0 => 20 * n_roots) */
    int precond;            /* dmrg_precond */
    int fp64_final;         /* 1: mixed modes report FP64 Rayleigh quotients <x|H|x>
                               (one FP64-arithmetic sigma per root after Davidson);
                               default 0 */
    int64_t mem_budget;     /* device bytes the plan may hold (0 => 90% of free) */
    int64_t scratch_bytes;  /* sigma GEMM scratch per chunk (0 => automatic) */
    int keep_envs;          /* 1: keep every bond's environment (sweeps) */
    int verbose;            /* 0 silent, 1 per-bond lines on stderr */
    int64_t tc_kchunk;      /* mixed modes: K-depth a sigma output tile accumulates in
                               FP32 tensor memory before it is added into the FP64
                               result (0 => default 1024); shorter chains cost more
                               FP64 atomics and lose less to FP32 accumulation */
    int fp64_store;         /* mixed modes: 1 = renormalise and form intermediates with the
                               FP64 engine and keep that FP64 operator store, plus its bf16
                               pieces for the tensor-core sigma (more memory and slower
                               renormalisation; the store then carries no tensor-core
                               accumulation error, and with fp64_final the energies are
                               Rayleigh quotients of the FP64 Hamiltonian); default 0 */
    int sigma_graph;        /* mixed modes: 1 = each sigma replays a CUDA graph (the split of
                               psi and the tensor-core launches) captured once per bond and
                               vector count, with psi / sigma staged through plan buffers;
                               default 1 */
    int sigma_tune;         /* mixed modes: 1 = the tile shape of the sigma work lists
                               (tile width 128 or 64, phase-2 K-chunk) is picked per bond by
                               timing each candidate on a sample of the bond's own work (every
                               8th output block, 16th beyond a million products, with all their
                               products); choices are cached by
                               the bond's sector-size histogram; ignored when tc_kchunk > 0
                               or sigma_tile_n > 0, and for lists of over 2^20 products (which
                               keep tile width 128 and the full K-chunk, the measured winner
                               there); default 1 */
    int sigma_tile_n;       /* mixed modes: 64 or 128 fixes the tile width of the sigma work
                               lists (no tuning); 0 = tuned or 128; default 0 */
    int refine;             /* mixed modes: 1 = FP64 residual correction of Davidson (a defect
                               correction, not in the paper, whose Davidson is FP64 throughout):
                               the mixed-precision Davidson runs until it meets tol or its
                               residual stalls at the mixed sigma's noise floor; then, per
                               outer round, the residual r = H x - theta x is formed with the
                               FP64-accurate sigma (dmrg_sigma_fp64: W = H X), and the next
                               inner mixed Davidson runs on P H_mixed P + W X^T + X W^T - X C X^T
                               (P = I - X X^T, C = sym(X^T W)), which equals H on X in both
                               directions; its Ritz vectors are X's corrections.  It stops when
                               the FP64 residual meets tol.  Energies are FP64 Rayleigh
                               quotients.  With fp64_store = 1 the result is that of the FP64
                               Hamiltonian; default 0 */
    int max_refine;         /* outer rounds of the residual correction (0 => 8) */
    int fp64_tc;            /* mixed modes with fp64_store = 1: the FP64 products (renormalisation,
                               intermediates, dmrg_sigma_fp64, the residual correction and FP64
                               Rayleigh quotients) run on the FP64-accurate tensor-core engine of
                               DMRG_FP64_TC instead of FP64 arithmetic units; default 0 */
    int host_tier;          /* dmrg_sweep (Sec. 2.3, the operators of blocks away from the
                               current bond kept off the GPU): 1 = every environment block
                               that the current and the next bond update do not read is kept
                               in pinned host memory only.  A block is copied out once, on a
                               copy stream, while the bond's Davidson runs (blocks never change
                               after they are built); the next bond's block is copied back on
                               the same stream, and the compute stream waits for it where it is
                               first used.  The arithmetic is that of host_tier = 0 on the same
                               data (FP64 sweeps agree bitwise).  A failed pinned allocation
                               returns DMRG_ENOMEM; default 0 */
    int sigma_per_term;     /* mixed modes, for measurement: 1 = the sigma work list is cut into
                               one scratch chunk per Hamiltonian term, i.e. a phase-1 and a
                               phase-2 launch per term (a launch-per-term baseline of the
                               grouped launch; Sec. 2.3 batches GEMMs per term); no tuning;
                               default 0 */
    double decim_tol32;     /* decimation eigensolver: off(rho)/|rho| at which the FP32 stage of
                               large density-matrix blocks hands over to the FP64 sweeps (it also
                               stops at the FP32 rounding floor); 0 => 1e-5 */
    int decim_fp64_units;   /* decimation eigensolver: 1 = the rotations of the FP64 sweeps that
                               follow the FP32 stage run on the FP64 units; 0 (default) = in
                               double-float arithmetic on the FP32 units (pairs of floats, ~48
                               significant bits; GB300 runs FP32 ~64x faster than FP64) */
} dmrg_options;

typedef struct {
    int64_t sigma_calls;          /* dmrg_sigma invocations (all vectors) */
    double sigma_flops;           /* algorithmic FLOPs of one sigma (current bond, one vector) */
    double sigma_ms_last;         /* device time of the last sigma call */
    double interm_flops;          /* FLOPs of forming the bond's intermediates */
    double renorm_flops_last;     /* FLOPs of the last renormalisation */
    double ms_interm, ms_gemm, ms_renorm, ms_davidson, ms_decim, ms_hdiag;
    int64_t n_terms;              /* sigma terms at the current bond */
    int64_t n_items;              /* (term x sector) GEMM items at the current bond */
    int64_t store_bytes;          /* operator store bytes of the current L and R */
    int64_t interm_bytes;         /* intermediate bytes at the current bond */
    int64_t device_bytes;         /* everything the plan holds on the device */
    int64_t kernel_launches;      /* kernels launched by the library since the plan was made */
    int64_t precond_fallbacks;    /* MLP -> Jacobi fallbacks */
    int davidson_iters_last;
    double ms_host_plan;          /* host time spent building work lists (all calls) */
    int64_t sigma_tiles[2];       /* mixed sigma: 128 x 128 output tiles of phase 1 / phase 2 */
    int64_t sigma_stages[2];      /* mixed sigma: 64-deep K stages of phase 1 / phase 2 */
    double sigma_mma_flops;       /* mixed sigma: tensor work of the tiles (one bf16 product) */
    int64_t sigma_maps;           /* mixed sigma: tensor maps of the current bond */
    double ms_decim_parts[4];     /* decimation: density matrices, eigensolver, host
                                     selection / new site tensor, next-bond guess (all calls) */
    int decim_sweeps_last;        /* block-Jacobi FP64 sweeps of the last decimation */
    double ms_sigma_dev;          /* device time of all completed sigma calls (CUDA events on
                                     the launching stream around each call) */
    double sigma_flops_dev;       /* algorithmic FLOPs of those calls (all vectors) */
    int64_t sigma_stages_dev;     /* mixed sigma: tensor-core K stages of those calls */
    int64_t sigma_timed;          /* number of sigma calls in ms_sigma_dev */
    double decim_conv_last[41];   /* last decimation: max over its matrices of off(rho)/|rho|
                                     before each eigensolver sweep (FP32 stage, then FP64) and
                                     at the end (0 after the last) */
    int decim_nmat_last;          /* last decimation: number of density-matrix blocks */
    int decim_nmax_last;          /* last decimation: largest block dimension */
    int decim_sweeps32_last;      /* last decimation: FP32 sweeps before the FP64 ones (0: FP64 only) */
    int sigma_tile_n;             /* mixed sigma: tile width of the current bond's work lists */
    int64_t sigma_kchunk;         /* mixed sigma: phase-2 K-chunk of the current bond */
    int64_t tunes;                /* autotuner runs (histograms not seen before) */
    int64_t tune_hits;            /* bonds whose histogram was already tuned */
    double ms_tune;               /* wall time of all autotuner runs */
    double tune_cand_ms[4];       /* last autotuner run: sample time per candidate
                                     (128 / K-chunk, 64 / K-chunk, 128 / half K-chunk, 64 / half) */
    double sigma_load_bytes[2][2];/* mixed sigma, one vector: operand bytes the tensor-core tiles
                                     load through TMA, [phase 1 / 2][other operands / phase-1
                                     scratch] (counts every box load, before any L2 reuse) */
    double renorm_flops_total;    /* algorithmic FLOPs of every renormalisation so far (products
                                     and their intermediates) */
    double interm_flops_total;    /* algorithmic FLOPs of forming every bond's intermediates */
    double davidson_rnorm_last;   /* last Davidson: largest residual 2-norm over the roots at exit
                                     (FP64-accurate residual when refine = 1) */
    int davidson_conv_last;       /* last Davidson: 1 if every root met tol */
    int davidson_stalled_last;    /* last Davidson (mixed): 1 if the mixed iteration stopped
                                     because its residual stalled at the noise floor */
    int davidson_refine_last;     /* last Davidson: residual-correction rounds (refine = 1) */
    int sigma_chunks;             /* scratch chunks (pairs of launches) of the current bond's sigma list */
    int64_t sigma_acc_calls;      /* FP64-accurate sigma calls (dmrg_sigma_fp64, refinement,
                                     FP64 Rayleigh quotients), all vectors */
    double ms_sigma_acc;          /* their device time */
    double sigma_acc_flops;       /* their algorithmic FLOPs */
    int64_t device_bytes_peak;    /* largest device_bytes since the plan was made */
    int64_t host_bytes;           /* pinned host memory held by the host tier */
    int64_t tier_out_bytes;       /* bytes copied device -> host by the host tier */
    int64_t tier_in_bytes;        /* bytes copied host -> device by the host tier */
    double ms_tier_wait;          /* host time spent waiting for host-tier copies to finish */
} dmrg_stats_t;

/* Default options: FP64, 1 root, tol 1e-6, 200 iterations, Jacobi. */
void dmrg_default_options(dmrg_options* opt);

/* Create a plan (Sec. 2.3: qops of a bond, Eq. Hsq integrals).
 *  h        K*K row-major one-electron integrals (host), copied.
 *  chol     n_chol > 0: n_chol*K*K Cholesky vectors L[X][p][q] (host), copied;
 *           the two-electron integrals are (pq|rs) = sum_X L[X][p][q] L[X][r][s],
 *           formed on the device.
 *           n_chol = 0: the full K*K*K*K array of chemist-notation integrals
 *           (pq|rs) at [((p*K + q)*K + r)*K + s] (host), copied; K <= 128; it
 *           must have the symmetry of real orbitals, (pq|rs) = (qp|rs) =
 *           (pq|sr) = (rs|pq) to 1e-12 of its largest entry (DMRG_EINVAL
 *           otherwise).
 *  e_core   constant energy added to reported energies.
 *  K,N,twoS orbitals, electrons, 2*Sz; N <= 2K, |twoS| <= min(N, 2K-N),
 *           N + twoS even.
 *  D        bond dimension used by dmrg_sweep when D_schedule is NULL.
 *  mps_path binary MPS file (format of synthetic_inputs.write_mps): sectors
 *           of every bond and block-sparse site tensors, left-orthonormal
 *           left of the centre, right-orthonormal right of centre+1.
 * Returns DMRG_EINVAL on inconsistent sizes or file, DMRG_ENUMERIC on a
 * non-finite integral, DMRG_EIO if the file is unreadable. */
dmrg_status dmrg_plan(const double* h, const double* chol, int n_chol, double e_core,
                      int K, int N, int twoS, int D, const dmrg_options* opt,
                      const char* mps_path, dmrg_plan_t* out);

/* Make bond (k, k+1) current (1 <= k <= K-1): renormalise (Eq. Renorm) the
 * left block of sites 1..k-1 and the right block of sites k+2..K from the
 * MPS, form the bond's intermediates (integral-weighted operator sums,
 * Sec. 2.2 "intermediates") and the sigma work list.  The MPS must be
 * left-orthonormal on 1..k-1 and right-orthonormal on k+2..K. */
dmrg_status dmrg_set_bond(dmrg_plan_t plan, int k, void* stream);

/* Canonical layout of the current bond (Sec. 2.1: the two-site wavefunction
 * Psi(L, c1, c2, R) is block-sparse in the (N, 2Sz) quantum numbers; one dense
 * d_l x d_r block, C order, per allowed (L, c1, c2, R), packed back to back).
 * dim = total length; n_sectors = number of sector blocks.  If offsets !=
 * NULL it receives n_sectors+1 offsets; if qn != NULL it receives 6 ints per
 * sector: (N_L, 2Sz_L, c1, c2, d_l, d_r).  Returns DMRG_EINVAL without a
 * current bond. */
dmrg_status dmrg_layout(dmrg_plan_t plan, int64_t* dim, int* n_sectors, int64_t* offsets, int* qn);

/* sigma = H psi (Eq. Sigma) for nvec vectors stored back to back (device,
 * FP64, canonical layout, length nvec*dim each).  psi and sigma must not
 * overlap.  Intermediate products go through the plan's scratch. */
dmrg_status dmrg_sigma(dmrg_plan_t plan, const double* psi_dev, double* sigma_dev, int nvec,
                       void* stream);

/* sigma = H psi evaluated in FP64 arithmetic over the plan's stored operators
 * (in the mixed modes the bf16 pieces are upcast exactly, hi + lo), on the
 * FP64 engine.  Separates the error of the mixed-precision products from the
 * rounding of the stored operators.  Same buffers as dmrg_sigma. */
dmrg_status dmrg_sigma_fp64(dmrg_plan_t plan, const double* psi_dev, double* sigma_dev, int nvec,
                            void* stream);

/* dmrg_sigma_fp64 on the FP64 arithmetic units even when the plan's FP64
 * products run on the FP64-accurate tensor-core engine (DMRG_FP64_TC, or
 * fp64_tc = 1): the plain FP64 GPU reference for the same stored operators.
 * Slow on GB300 (~1 TFLOP/s of FP64); same buffers as dmrg_sigma. */
dmrg_status dmrg_sigma_fp64_units(dmrg_plan_t plan, const double* psi_dev, double* sigma_dev, int nvec,
                                  void* stream);

/* Same as dmrg_sigma with HOST buffers (copies to and from the device inside;
 * the end-to-end path of the benchmark). */
dmrg_status dmrg_sigma_host(dmrg_plan_t plan, const double* psi_host, double* sigma_host,
                            int nvec, void* stream);

/* Diagonal of H_eff at the current bond (device, FP64, canonical layout). */
dmrg_status dmrg_hdiag(dmrg_plan_t plan, double* diag_dev, void* stream);

/* Davidson (Sec. 2.1) for the lowest n_roots eigenpairs at the current bond.
 *  psi_dev  in: n_roots guesses, out: Ritz vectors (device, FP64).
 *  energies out (host): n_roots eigenvalues + e_core.
 *  iters    out (host): iterations used (may be NULL).
 *  precond  dmrg_precond; MLP falls back to Jacobi (counted in stats) if its
 *           correction is not finite or not a descent direction.
 * Returns DMRG_ENOTCONV if max_iter is reached above tol (energies filled). */
dmrg_status dmrg_davidson(dmrg_plan_t plan, double* psi_dev, int n_roots, double tol, int max_iter,
                          int precond, double* energies, int* iters, void* stream);

/* Switch the FP64 residual correction of later dmrg_davidson calls (the
 * refine / max_refine options; mixed modes only).  DMRG_EINVAL for a negative
 * max_refine. */
dmrg_status dmrg_set_refine(dmrg_plan_t plan, int refine, int max_refine);

/* One two-site bond update (Sec. 2.1, Fig. flowchart) from HOST buffers, the
 * end-to-end path of a caller that keeps its vectors in host memory:
 *  psi_host   n_roots guesses of the current bond (host, FP64, canonical
 *             layout, n_roots x dim), copied to the device.
 * Davidson (as dmrg_davidson with the plan's tol, max_iter and precond), then
 * decimation to D (as dmrg_decimate, forward or backward), which makes the next
 * bond current; its guess is copied back.
 *  energies   out (host): n_roots energies (+ e_core).
 *  iters      out (host, may be NULL): Davidson iterations.
 *  discarded  out (host, may be NULL): discarded weight.
 *  next_psi_host  out (host, may be NULL): the next bond's guess.
 *  next_dim   in: capacity of next_psi_host in elements per root (0 if NULL);
 *             out: the next bond's vector length.  The guess is copied only
 *             when the capacity suffices.
 * Returns DMRG_ENOTCONV (after decimating) if Davidson stopped above tol. */
dmrg_status dmrg_update_bond_host(dmrg_plan_t plan, const double* psi_host, int n_roots, int D, int forward,
                                  double* energies, int* iters, double* discarded, double* next_psi_host,
                                  int64_t* next_dim, void* stream);

/* Decimation (Sec. 2.1): truncate the current bond's two-site vectors psi_dev
 * (n_roots of them; state-averaged density matrix if > 1) to at most D states
 * (largest density-matrix eigenvalues, ties by sector order then rank), update
 * A[k] (forward) or A[k+1] (backward), renormalise the grown block and make the
 * next bond (k+1 or k-1) current.
 *  discarded     out: sum of the dropped eigenvalues.
 *  next_dim      in: capacity of next_psi_dev in elements per root (0 if
 *                next_psi_dev is NULL); out: length of the next bond's vector.
 *  next_psi_dev  receives the guess for the next bond (U^T psi A[k+2] or
 *                A[k-1] psi V) when the capacity suffices. */
dmrg_status dmrg_decimate(dmrg_plan_t plan, const double* psi_dev, int n_roots, int D, int forward,
                          double* discarded, double* next_psi_dev, int64_t* next_dim, void* stream);

/* Two-dot sweeps from bond (1,2): forward over bonds 1..K-2 then backward over
 * K-1..2 (Sec. 2.3).  energies[s], discarded[s]: lowest energy at the last bond
 * and largest discarded weight of sweep s.  D_schedule (may be NULL) gives the
 * bond dimension of each sweep. */
dmrg_status dmrg_sweep(dmrg_plan_t plan, int n_sweeps, const int* D_schedule, double* energies,
                       double* discarded, void* stream);

/* Linear extrapolation of energies to zero discarded weight (Tab. energy and
 * Fig. extrapolation: E(w) = A w + E_{w=0}, fitted by least squares over a
 * series of runs, e.g. the energies and discarded weights that dmrg_sweep
 * returns for a D schedule).
 *  w, E    n host values each: discarded weights and energies (Eh); read only.
 *  n       number of points, >= 2.
 *  e0      out: E_{w=0}, the intercept.
 *  slope   out (may be NULL): A.
 *  rms     out (may be NULL): root-mean-square residual of the fit.
 * Host arithmetic only: no plan, no device work, callable without a GPU.
 * DMRG_EINVAL for n < 2, a NULL w / E / e0, non-finite values, or weights that
 * are all equal. */
dmrg_status dmrg_extrapolate(const double* w, const double* E, int n, double* e0, double* slope, double* rms);

/* Write the current MPS (Sec. 2.1: the site tensors after the decimations
 * so far, left-orthonormal left of the centre and right-orthonormal right of
 * it) in the format of the input file.  DMRG_EIO if the file cannot be
 * written. */
dmrg_status dmrg_save_mps(dmrg_plan_t plan, const char* path);

/* Copy the plan's counters (dmrg_stats_t above: phase times, algorithmic
 * FLOPs of sigma (Tab. stat counts its GEMMs the same way), renormalisation
 * and intermediates, bytes held, launches, solver histories) into *out. */
dmrg_status dmrg_stats(dmrg_plan_t plan, dmrg_stats_t* out);

/* One-line description of the last error of this plan (or of plan creation
 * if plan is NULL).  The string is owned by the library. */
const char* dmrg_last_error(dmrg_plan_t plan);

void dmrg_destroy(dmrg_plan_t plan);

/* ------------------------------------------------------------------------
 * Learned Davidson preconditioner (DMRG_PRECOND_MLP).  Not in the paper.
 * A per-element MLP g(x), 5 -> 64 -> 64 -> 1 with tanh, scales the diagonal
 * correction: t_i = -g_i r_i / (H_ii - theta).  Inputs of element i:
 * ((H_ii - theta)/s, theta/s, r_i/|r|_inf, N_L/N, 2Sz_L/N), s = max|H_ii - theta|.
 * FP32 parameters (Adam), bf16 weights in the Davidson inference.  Until it is
 * trained (or when an output is not finite) Davidson uses the Jacobi step and
 * counts the fallback in dmrg_stats_t.precond_fallbacks.
 * ------------------------------------------------------------------------ */

/* Seeded initialisation (g = 1, i.e. the Jacobi step); clears "trained". */
dmrg_status dmrg_mlp_init(dmrg_plan_t plan, uint32_t seed);

/* Runs plain (Jacobi) Davidson at the current bond from psi_dev (updated to
 * the Ritz vector); at every iteration the Jacobi-Davidson correction
 * equation of root 0 is solved by MINRES (jd_iters iterations at most), and
 * up to per_solve strided elements give training pairs (features, target
 * g_i = -t_i (H_ii - theta)/r_i, clipped to [-10, 10], weight
 * (r_i / (H_ii - theta))^2 scaled to mean 1 over the solve: the weighted
 * squared error of g is the squared error of the correction t) appended to
 * the plan's training set.  *n_pairs receives the number added. */
dmrg_status dmrg_mlp_harvest(dmrg_plan_t plan, double* psi_dev, int max_iter, int jd_iters, int64_t per_solve,
                             double* energy, int64_t* n_pairs, void* stream);

/* steps Adam steps (learning rate lr) on batches of `batch` pairs drawn from
 * the first nine tenths of the training set by a seeded counter-based
 * generator; the last tenth (the latest solves) is held out.  Loss = weighted
 * mean squared error of g (weights of dmrg_mlp_harvest).  Out (host, each may
 * be NULL): loss of the first and last training batch, loss of the held-out
 * pairs before and after training (0 with fewer than 20 pairs).  Marks the
 * network trained. */
dmrg_status dmrg_mlp_train(dmrg_plan_t plan, int steps, int64_t batch, float lr, uint64_t seed,
                           float* loss_first, float* loss_last, float* held_first, float* held_last,
                           void* stream);

/* g_dev[i] = g(x_dev[5i .. 5i+4]) for n rows (device FP32); bf16 selects the
 * inference weights. */
dmrg_status dmrg_mlp_eval(dmrg_plan_t plan, const float* x_dev, int64_t n, float* g_dev, int bf16, void* stream);

/* Gradient of (1/n) sum_i w_i (g(x_i) - y_i)^2 with respect to the parameters
 * (layout of dmrg_mlp_params) into grad_dev, the loss into loss_dev (device);
 * w_dev may be NULL (all weights 1). */
dmrg_status dmrg_mlp_gradient(dmrg_plan_t plan, const float* x_dev, const float* y_dev, const float* w_dev,
                              int64_t n, float* grad_dev, float* loss_dev, void* stream);

/* Parameters (host, dmrg_mlp_num_params() floats: W1[64x5], b1[64],
 * W2[64x64], b2[64], W3[64], b3): get (set = 0) or set (set = 1; marks the
 * network trained). */
dmrg_status dmrg_mlp_params(dmrg_plan_t plan, float* host, int set);
int dmrg_mlp_num_params(void);

/* ------------------------------------------------------------------------
 * Kernel-level entry point used by the unit tests (the same grouped GEMM
 * engine that runs every sigma, renormalisation and intermediate product).
 * Computes, for each of n_out output blocks o (host arrays of n_out):
 *   C_o (m_o x n_o, row-major at c + c_off[o], ld n_o)
 *       = sum over segments s in [seg_beg[o], seg_beg[o+1]) of
 *         alpha[s] * op(A_s) * op(B_s)
 * where A_s is m_o x k[s] at a + a_off[s] (row-major ld lda[s], or its
 * transpose if a_tr[s]) and B_s is k[s] x n_o at b + b_off[s] (ld ldb[s], or
 * transposed if b_tr[s]).  a, b, c are device FP64 buffers.  precision
 * selects the FP64 engine (DMRG_FP64), the FP64-accurate tensor-core engine
 * (DMRG_FP64_TC) or the bf16 tensor-core engine (operands are split into bf16
 * hi/lo on the device for BF16X3).
 * ------------------------------------------------------------------------ */
dmrg_status dmrg_grouped_gemm(int precision, int n_out, const int* m, const int* n,
                              const int64_t* c_off, const int* seg_beg, const int* k,
                              const int64_t* a_off, const int* lda, const int* a_tr,
                              const int64_t* b_off, const int* ldb, const int* b_tr,
                              const double* alpha, const double* a, const double* b, double* c,
                              void* stream);

/* ------------------------------------------------------------------------
 * Allocation-free variant of dmrg_grouped_gemm with precision DMRG_FP64.
 * The paper has no counterpart: this exists for callers that cannot obtain
 * device memory when they need the product (a process whose memory is all
 * held by its own pool, or one that must not pay the device-wide
 * synchronisation of cudaFree between overlapped streams).
 *
 * Arguments, layouts and results are those of dmrg_grouped_gemm (FP64): C
 * is overwritten block by block (blocks with no segment are set to zero), so
 * nothing has to start at zero.  a, b, c are caller-owned device FP64
 * buffers; the host arrays are read before the call returns.
 *
 * The work list (48 bytes per 64 x 64 output tile plus 40 per segment,
 * tile list padded to 256 bytes) is copied into a fixed static device array
 * of dmrg_noalloc_scratch_bytes() bytes (4 MiB); larger lists are rejected
 * with DMRG_EINVAL and a message giving the size needed.  No device memory is
 * allocated or freed.
 *
 * The kernel runs asynchronously on `stream` (launch errors are returned;
 * faults surface at the caller's next synchronisation), but the work list is
 * copied from pageable host memory, which may make the call wait for the
 * stream's earlier work before it returns.  Because that host copy does not
 * outlive the call, a stream that is being captured is refused with
 * DMRG_EINVAL before anything is enqueued.  The first call on a device
 * looks up the array's device address with that device current (with lazy
 * module loading the driver also places the array in device memory at that
 * point); make it before any stream capture begins.  All calls share the one array: calls on
 * one stream are ordered, but calls whose executions overlap (different
 * streams, or threads without ordering) race on it and must be serialised by
 * the caller.
 * ------------------------------------------------------------------------ */
dmrg_status dmrg_grouped_gemm_noalloc(int n_out, const int* m, const int* n, const int64_t* c_off,
                                      const int* seg_beg, const int* k, const int64_t* a_off,
                                      const int* lda, const int* a_tr, const int64_t* b_off,
                                      const int* ldb, const int* b_tr, const double* alpha,
                                      const double* a, const double* b, double* c, void* stream);

/* Size in bytes of the static work-list array of dmrg_grouped_gemm_noalloc. */
int64_t dmrg_noalloc_scratch_bytes(void);

/* Check of the bounded device waits every warp-specialised kernel of the
 * library uses (mbarrier waits that give up after a time limit and set a device
 * error word instead of spinning forever).  One CTA initialises an mbarrier,
 * arrives on it only if `arrive` is nonzero, and waits on it for at most
 * `seconds` (0 < seconds <= 2) with the kernels' wait routine; no copy or MMA is
 * in flight.  Returns DMRG_OK if the wait completed, DMRG_ETIMEOUT if it gave up
 * (the status the library's kernels report through their error words), and
 * leaves the context usable either way.  DMRG_EINVAL for seconds outside the
 * range.  Synchronises the stream. */
dmrg_status dmrg_selftest_wait(double seconds, int arrive, void* stream);

/* Library build / device information: writes a short string. */
const char* dmrg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DMRG_H */

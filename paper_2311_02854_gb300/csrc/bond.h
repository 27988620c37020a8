// Functions of bond.cu / solver.cu shared with the C-ABI layer.
#pragma once

#include "plan.h"

namespace dmrg {

// offsets of the intermediates in their store (what the sigma lists refer to)
void interm_bases(Interms& im, const Block* blocks[2]);
// bases_set: interm_bases already ran for im (im is then only read)
void form_interms(Plan& P, Interms& im, const Block* blocks[2], IntermStore& S, double& flops,
                  bool bases_set = false);
void free_interms(Plan& P, IntermStore& S);
void free_block(Plan& P, std::unique_ptr<Block>& b);
void ensure_ident(Plan& P, int n);
void ensure_scratch(Plan& P, int64_t n);      // scratch of the plan's engine
void ensure_scratch_f64(Plan& P, int64_t n);  // FP64 scratch (FP64 engine in either mode)
int64_t scratch_cap(const Plan& P);      // scratch elements of the plan's engine
int64_t scratch_cap_f64(const Plan& P);  // scratch elements of FP64-engine lists
std::unique_ptr<Block> make_vacuum(Plan& P, bool right_end);
Basis bond_basis(const Plan& P, int b, bool right_side);
std::unique_ptr<Block> renormalise(Plan& P, const Block& X, int m, bool forward);
void ensure_env(Plan& P, int k);
void build_layout(Plan& P, int k);
void set_bond(Plan& P, int k);
BufTable bond_buffers(Plan& P, const double* psi, double* out);
// sigma with the plan's engine (tensor cores in mixed precision)
void sigma(Plan& P, const double* psi, double* out, int nvec, cudaStream_t st);
// sigma in FP64 arithmetic over the stored operators (either precision)
void sigma_fp64(Plan& P, const double* psi, double* out, int nvec, cudaStream_t st);
// the same on the FP64 arithmetic units, whatever engine the plan's FP64 products use
void sigma_fp64_units(Plan& P, const double* psi, double* out, int nvec, cudaStream_t st);
void hdiag(Plan& P, double* out, cudaStream_t st);

// tier.cu: environment blocks in pinned host memory between their uses
void tier_out(Plan& P, Block& b);   // start the eviction of a resident block
void tier_in(Plan& P, Block& b);    // start bringing an evicted block back (prefetch)
void tier_need(Plan& P, Block& b);  // the block is used next on P.stream
void tier_drain(Plan& P, bool wait);  // free the device arrays of evictions whose copies are done
                                      // (wait: wait for every copy first)
void tier_release(Plan& P, Block& b);  // before a block is freed
void tier_destroy(Plan& P);
// evict every block that the bond k update and the next bond do not use, and
// prefetch the next bond's block (forward: right[k+2], backward: left[k-2])
void tier_policy(Plan& P, int k, bool forward);

// solver.cu
dmrg_status davidson(Plan& P, double* psi, int n_roots, double tol, int max_iter, int precond,
                     double* energies, int* iters);
void decimate(Plan& P, const double* psi, int n_roots, int D, bool forward, double* discarded);
void two_site_guess(Plan& P, double* out);
dmrg_status sweep(Plan& P, int n_sweeps, const int* D_schedule, double* energies, double* discarded);

}  // namespace dmrg

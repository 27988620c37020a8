// Tensor-core (tcgen05, sm_103a) segmented grouped GEMM on bf16 operand pieces.
#pragma once

#include <cuda_bf16.h>

#include "engine.h"

namespace dmrg {

// Output modes of the tensor-core engine (Tile::mode)
enum TcMode : uint8_t {
    TC_ATOMIC_F64 = 2,   // atomicAdd(double) of alpha * acc
    TC_STORE_SPLIT = 3,  // store alpha * acc as bf16 pieces (hi, lo) with the same offsets
    TC_ATOMIC_F32 = 4,   // atomicAdd(float)
    TC_STORE_F32 = 5,
};

// Operands: every buffer id holds `nsplit` bf16 pieces with identical layouts
// (x ~ hi + lo).  A segment's A / B are K-major (tr = 0) or MN-major (tr = 1).
struct TcBufs {
    const __nv_bfloat16* hi[kMaxBufs];
    const __nv_bfloat16* lo[kMaxBufs];
    int64_t vstride[kMaxBufs];
    void* out[kMaxBufs];       // double* / float* / bf16 hi pieces (by mode)
    void* out_lo[kMaxBufs];    // bf16 lo pieces for TC_STORE_SPLIT
    int64_t out_vstride[kMaxBufs];
    int* counter;              // dynamic tile counter (zeroed before each launch)
    int* err;                  // device error word (0 = ok)
};

// Launch over the tiles of `w` (Seg::alpha must be +1 or -1: a sign applied
// through the MMA negate bit; Tile::alpha scales the epilogue).
void launch_seg_gemm_tc(const WorkList& w, const TcBufs& b, int nvec, int nsplit, cudaStream_t st);

int tc_num_sms();

// FP64 (unpadded rows of length n, ld_src) -> bf16 pieces (rows padded to ld_dst)
void dev_split_f64(const double* src, int64_t rows, int n, int64_t ld_src, __nv_bfloat16* hi,
                   __nv_bfloat16* lo, int64_t ld_dst, cudaStream_t st);
// FP32 -> bf16 pieces, same layout, n elements
void dev_split_f32(const float* src, int64_t n, __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t st);
// batched block copy FP64 -> pieces: for each job (src_off, dst_off, rows, cols, ld_src, ld_dst)
struct SplitJob {
    int64_t src_off, dst_off;
    int rows, cols, ld_src, ld_dst;
};
void dev_split_blocks(const double* src, const SplitJob* d_jobs, int njobs, __nv_bfloat16* hi, __nv_bfloat16* lo,
                      cudaStream_t st);

}  // namespace dmrg

// Tensor-core segmented grouped GEMM for sm_103a (5th-generation tensor cores):
// operands staged in shared memory (128B-swizzled canonical layouts, K-major
// or MN-major), tcgen05.mma kind::f16 with bf16 inputs and FP32 accumulation
// in tensor memory, completion tracked by mbarriers, persistent
// warp-specialised CTAs (one per SM) walking the tiles round-robin, the
// vectors of a launch innermost (the copies of one tile for every vector run
// back to back on neighbouring CTAs, so that the operator boxes they share are
// read from DRAM once and then served from L2).  One output
// tile (128 x 128) accumulates the K-segments of its block (the term sum of
// the sigma reduction happens in the accumulator).  bf16 "pieces": an operand x is held as hi + lo; with
// nsplit = 2 each product runs as hi*hi + hi*lo + lo*hi.
#include <cuda_bf16.h>

#include <algorithm>

#include "ptx.h"
#include "tc.h"

namespace dmrg {
namespace {

using namespace ptx;

constexpr int TM = 128, TN = 128, TK = 64;
static_assert(sizeof(Tile) % 4 == 0 && sizeof(TSeg) % 4 == 0, "work-list records are moved by 32-bit shuffles");
static_assert(sizeof(TSeg) % 16 == 0, "segment records stay 16-byte aligned");
constexpr int PIECE_BYTES = TM * TK * 2;  // one 128 x 64 bf16 operand tile
constexpr uint32_t TMEM_COLS = 128;

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// instruction descriptor of a full 128 x 128 tile
__device__ __forceinline__ uint32_t idesc(int a_mn, int b_mn, int neg) { return idesc_mn(a_mn, b_mn, neg, TN, TM); }

// Stage one 128 x 64 (M x K) operand piece into shared memory in the 128B-swizzled
// canonical layout the MMA descriptors describe.  Element (r, k) of the
// operand is base[r*ld + k] (mn = 0: K-major) or base[k*ld + r] (mn = 1:
// MN-major), valid for r < R, k < K; chunks outside are zero-filled (no global
// read).  Producer thread p always handles the same 16-byte column chunk of 8
// rows 16 (K-major) or 8 (MN-major) apart, so the swizzle and the validity of
// the chunk's columns are loop invariant and each copy costs a few instructions.
__device__ __forceinline__ void load_piece(uint32_t sdst, const __nv_bfloat16* base, int ld, int mn, int r0, int R,
                                           int k0, int K, int p) {
    if (!mn) {
        const int c = p & 7, rr = p >> 3;  // chunk, first row (0..15)
        const int kk = k0 + c * 8;
        const int cvalid = kk < K ? min(8, K - kk) * 2 : 0;
        uint32_t dst = sdst + (uint32_t)((rr >> 3) * 1024 + (rr & 7) * 128 + ((c ^ (rr & 7)) << 4));
        const __nv_bfloat16* src = base + (int64_t)(r0 + rr) * ld + kk;
        const int64_t step = (int64_t)16 * ld;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool ok = (r0 + rr + 16 * j < R) && cvalid > 0;
            cp_async16(dst, ok ? (const void*)src : (const void*)base, ok ? cvalid : 0);
            dst += 2048;
            src += step;
        }
    } else {
        const int c = p & 15, kr = p >> 4;  // chunk along M, first K row (0..7)
        const int rr = r0 + c * 8;
        const int cvalid = rr < R ? min(8, R - rr) * 2 : 0;
        uint32_t dst = sdst + (uint32_t)((c >> 3) * 1024 + kr * 128 + (((c & 7) ^ kr) << 4));
        const __nv_bfloat16* src = base + (int64_t)(k0 + kr) * ld + rr;
        const int64_t step = (int64_t)8 * ld;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool ok = (k0 + kr + 8 * j < K) && cvalid > 0;
            cp_async16(dst, ok ? (const void*)src : (const void*)base, ok ? cvalid : 0);
            dst += 2048;
            src += step;
        }
    }
}

__device__ __forceinline__ void cp_async_wait_n(int n) {
    // wait until at most n committed groups are pending (n is 0..2 here)
    if (n <= 0) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    else if (n == 1) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    else asm volatile("cp.async.wait_group 2;\n" ::: "memory");
}
// Roles of the persistent kernel (one CTA per SM):
//   warps 0-3  epilogue: TMEM -> registers -> global (warp w owns TMEM lanes 32w..32w+31)
//   warps 4-7  producers: cp.async of the operand pieces of each 64-deep K stage
//   warp  8    MMA issuer (lane 0): tcgen05.mma into one of two TMEM accumulators
// Stages flow through a ring of STAGES shared-memory slots (full / empty
// mbarriers); tiles alternate between two 128-column TMEM accumulators
// (tmem_full / tmem_empty), so loads of the next stages, the MMAs of one tile
// and the epilogue of the previous tile overlap.  Every wait is bounded; on a
// timeout the CTA sets the error word and winds down.
constexpr int kEpiWarps = 4, kProdWarps = 4;
constexpr int NPROD = kProdWarps * 32;
constexpr int THREADS2 = (kEpiWarps + kProdWarps + 1) * 32;
template <int NSPLIT>
struct Cfg2 {
    static constexpr int STAGES = (NSPLIT == 1) ? 6 : (NSPLIT == 2 ? 3 : 2);
    static constexpr int STAGE_BYTES = 2 * NSPLIT * PIECE_BYTES;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
    // the producers publish a stage's full barrier LAG stages after issuing it
    static constexpr int LAG = STAGES - 1 < 2 ? STAGES - 1 : 2;
};

// Piece products of a split-precision MMA: x = sum_i x_i with |x_i| ~ 2^-8i |x|;
// products x_i y_j with i + j <= NSPLIT - 1 are kept (1, 3 or 6 of them).
template <int NSPLIT>
struct Prods {
    static constexpr int N = NSPLIT == 1 ? 1 : (NSPLIT == 2 ? 3 : 6);
};
__device__ __forceinline__ int prod_a(int pr) { return (0x210100 >> (4 * pr)) & 0xF; }  // 0,0,1,0,1,2
__device__ __forceinline__ int prod_b(int pr) { return (0x012010 >> (4 * pr)) & 0xF; }  // 0,1,0,2,1,0

struct StageMeta {
    uint8_t a_mn, b_mn, neg, flags;  // flags: 1 first stage of a tile, 2 last, 4 no MMA (empty tile)
    int32_t k16;                     // 16-deep MMA steps holding data (1..4)
};

__device__ __forceinline__ int tile_stages(const Tile& T, const Seg* __restrict__ segs) {
    int nst = 0;
    for (int s = T.seg_beg; s < T.seg_end; ++s) nst += (segs[s].k + TK - 1) / TK;
    return nst;
}

// Epilogue of one tile by warps 0-3 (warp w owns TMEM lanes / tile rows
// 32w..32w+31): accumulator columns at TMEM address tacc -> registers, release
// of the accumulator (one arrive per warp on `tempty`), then alpha * acc
// written or accumulated into the output in the tile's mode.
template <int NSPLIT>
__device__ __forceinline__ void epilogue_tile(const Tile& T, int v, int nst, uint32_t tacc, int warp, int lane,
                                              const TcBufs& B, uint32_t tempty) {
    const int row = warp * 32 + lane;
    const int r = T.m0 + row;
    const bool rok = r < T.m;
    const float alpha = T.alpha;
    uint32_t acc[TN];
    if (nst > 0) {
#pragma unroll
        for (int cg = 0; cg < TN / 32; ++cg) {
            uint32_t (&a32)[32] = *reinterpret_cast<uint32_t(*)[32]>(&acc[cg * 32]);
            tmem_ld32(tacc + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cg * 32), a32);
        }
        tmem_wait_ld();
    } else {
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[j] = 0u;
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(tempty);
    if (!rok || (nst == 0 && (T.mode == TC_ATOMIC_F64 || T.mode == TC_ATOMIC_F32))) return;
    const int ncol = min(T.tn > 0 ? T.tn : TN, T.n - T.n0);  // the FP64-engine work list leaves tn 0
    const int64_t off = T.c_off + (int64_t)r * T.ldc + T.n0 + (int64_t)v * B.out_vstride[T.c_buf];
    if (T.mode == TC_ATOMIC_F64) {
        double* o = (double*)B.out[T.c_buf] + off;
#pragma unroll
        for (int j = 0; j < TN; ++j)
            if (j < ncol) atomicAdd(o + j, (double)alpha * (double)__uint_as_float(acc[j]));
    } else if (T.mode == TC_ATOMIC_F32) {
        float* o = (float*)B.out[T.c_buf] + off;
#pragma unroll
        for (int j = 0; j < TN; ++j)
            if (j < ncol) atomicAdd(o + j, alpha * __uint_as_float(acc[j]));
    } else if (T.mode == TC_STORE_F32) {
        float* o = (float*)B.out[T.c_buf] + off;
#pragma unroll
        for (int j = 0; j < TN; ++j)
            if (j < ncol) o[j] = alpha * __uint_as_float(acc[j]);
    } else {  // TC_STORE_SPLIT: chunks of 8 (rows padded to multiples of 8)
        __nv_bfloat16* oh = (__nv_bfloat16*)B.out[T.c_buf] + off;
        __nv_bfloat16* ol = (__nv_bfloat16*)B.out_lo[T.c_buf] + off;
#pragma unroll
        for (int j0 = 0; j0 < TN; j0 += 8) {
            if (j0 >= ncol) break;
            __align__(16) __nv_bfloat16 h8[8], l8[8], m8[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float x = alpha * __uint_as_float(acc[j0 + j]);
                const __nv_bfloat16 h = __float2bfloat16_rn(x);
                h8[j] = h;
                const float r = x - __bfloat162float(h);
                l8[j] = __float2bfloat16_rn(r);
                m8[j] = __float2bfloat16_rn(r - __bfloat162float(l8[j]));
            }
            *(uint4*)(oh + j0) = *(const uint4*)h8;
            if (NSPLIT >= 2) *(uint4*)(ol + j0) = *(const uint4*)l8;
            if (NSPLIT == 3) *(uint4*)(ol + B.out_pstride[T.c_buf] + j0) = *(const uint4*)m8;
        }
    }
}

template <int NSPLIT>
__global__ void __launch_bounds__(THREADS2, 1)
    tc_seg_gemm_kernel(const Tile* __restrict__ tiles, int ntiles, int nvec, const Seg* __restrict__ segs, TcBufs B) {
    using C = Cfg2<NSPLIT>;
    constexpr int S = C::STAGES;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[S], empty_bar[S], tfull_bar[2], tempty_bar[2], drain_bar;
    __shared__ StageMeta meta[S];
    __shared__ uint32_t tmem_base_s;
    __shared__ int fail_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_base_s)),
                     "r"(2 * TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&full_bar[s]), NPROD);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&tfull_bar[b]), 1);
            mbar_init(smem_u32(&tempty_bar[b]), kEpiWarps);
        }
        mbar_init(smem_u32(&drain_bar), 1);
        fail_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;
    const int total = ntiles * nvec;
    bool failed = false;

    if (warp >= kEpiWarps && warp < kEpiWarps + kProdWarps) {
        // ---------------- producers ----------------
        const int p = tid - kEpiWarps * 32;
        uint32_t q = 0;
        auto finish_stage = [&](uint32_t qs) {  // stage qs's copies are complete: publish it
            fence_proxy_async();
            mbar_arrive(smem_u32(&full_bar[qs % S]));
        };
        auto begin_stage = [&](uint32_t qs) -> bool {  // wait until slot of stage qs is free
            if (qs >= (uint32_t)S && !mbar_wait(smem_u32(&empty_bar[qs % S]), ((qs / S) - 1) & 1u)) return false;
            return true;
        };
        constexpr int LAG = C::LAG;
        auto end_issue = [&]() {  // after committing stage q: publish stage q - LAG
            cp_async_commit();
            if (q >= (uint32_t)LAG) {
                cp_async_wait_n(LAG);
                finish_stage(q - LAG);
            }
            ++q;
        };
        for (int t = blockIdx.x; t < total && !failed; t += gridDim.x) {
            const int tix = t / nvec, v = t % nvec;
            const Tile T = tiles[tix];
            const int nst = tile_stages(T, segs);
            if (nst == 0) {
                if (!begin_stage(q)) { failed = true; break; }
                if (p == 0) meta[q % S] = StageMeta{0, 0, 0, 1 | 2 | 4, 0};
                end_issue();
                continue;
            }
            int done = 0;
            for (int s = T.seg_beg; s < T.seg_end && !failed; ++s) {
                const Seg Sg = segs[s];
                const int a_mn = Sg.a_tr ? 1 : 0, b_mn = Sg.b_tr ? 0 : 1;
                const int64_t ao = Sg.a_off + (int64_t)v * B.vstride[Sg.a_buf];
                const int64_t bo = Sg.b_off + (int64_t)v * B.vstride[Sg.b_buf];
                for (int k0 = 0; k0 < Sg.k; k0 += TK) {
                    if (!begin_stage(q)) { failed = true; break; }
                    const uint32_t sa = sbase + (q % S) * C::STAGE_BYTES;
                    const uint32_t sb = sa + NSPLIT * PIECE_BYTES;
                    load_piece(sa, B.hi[Sg.a_buf] + ao, Sg.lda, a_mn, T.m0, T.m, k0, Sg.k, p);
                    load_piece(sb, B.hi[Sg.b_buf] + bo, Sg.ldb, b_mn, T.n0, T.n, k0, Sg.k, p);
                    if (NSPLIT >= 2) {
                        load_piece(sa + PIECE_BYTES, B.lo[Sg.a_buf] + ao, Sg.lda, a_mn, T.m0, T.m, k0, Sg.k, p);
                        load_piece(sb + PIECE_BYTES, B.lo[Sg.b_buf] + bo, Sg.ldb, b_mn, T.n0, T.n, k0, Sg.k, p);
                    }
                    if (NSPLIT == 3) {
                        load_piece(sa + 2 * PIECE_BYTES, B.lo[Sg.a_buf] + B.pstride[Sg.a_buf] + ao, Sg.lda, a_mn, T.m0,
                                   T.m, k0, Sg.k, p);
                        load_piece(sb + 2 * PIECE_BYTES, B.lo[Sg.b_buf] + B.pstride[Sg.b_buf] + bo, Sg.ldb, b_mn, T.n0,
                                   T.n, k0, Sg.k, p);
                    }
                    if (p == 0) {
                        const int kv = min(TK, Sg.k - k0);
                        meta[q % S] = StageMeta{(uint8_t)a_mn, (uint8_t)b_mn, (uint8_t)(Sg.alpha < 0.0 ? 1 : 0),
                                                (uint8_t)((done == 0 ? 1 : 0) | (done == nst - 1 ? 2 : 0)),
                                                (kv + 15) / 16};
                    }
                    end_issue();
                    ++done;
                }
            }
        }
        // publish the last LAG stages (or wind down after a failure)
        cp_async_wait0();
        for (uint32_t qs = (q >= (uint32_t)LAG ? q - LAG : 0); qs < q; ++qs) finish_stage(qs);
    } else if (warp == kEpiWarps + kProdWarps) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            uint32_t q = 0, tc = 0;
            for (int t = blockIdx.x; t < total && !failed; t += gridDim.x, ++tc) {
                const uint32_t buf = tc & 1u, use = tc >> 1;
                if (use > 0 && !mbar_wait(smem_u32(&tempty_bar[buf]), (use - 1) & 1u)) { failed = true; break; }
                tc_fence_after();
                const uint32_t dt = tmem + buf * TMEM_COLS;
                for (;;) {
                    const uint32_t slot = q % S;
                    if (!mbar_wait(smem_u32(&full_bar[slot]), (q / S) & 1u)) { failed = true; break; }
                    tc_fence_after();
                    const StageMeta M = meta[slot];
                    if (!(M.flags & 4)) {
                        const uint32_t sa = sbase + slot * C::STAGE_BYTES;
                        const uint32_t sb = sa + NSPLIT * PIECE_BYTES;
                        const uint32_t id = idesc(M.a_mn, M.b_mn, M.neg);
                        for (int kk = 0; kk < M.k16; ++kk) {
#pragma unroll
                            for (int pr = 0; pr < Prods<NSPLIT>::N; ++pr) {
                                const int pa = prod_a(pr), pb = prod_b(pr);
                                const uint32_t a_s = sa + pa * PIECE_BYTES;
                                const uint32_t b_s = sb + pb * PIECE_BYTES;
                                const uint64_t ad =
                                    M.a_mn ? sdesc(a_s + kk * 4096, 1024, 2048) : sdesc(a_s + kk * 32, 16, 1024);
                                const uint64_t bd =
                                    M.b_mn ? sdesc(b_s + kk * 4096, 1024, 2048) : sdesc(b_s + kk * 32, 16, 1024);
                                const uint32_t acc = ((M.flags & 1) && kk == 0 && pr == 0) ? 0u : 1u;
                                mma_bf16(dt, ad, bd, id, acc);
                            }
                        }
                    }
                    mma_commit(smem_u32(&empty_bar[slot]));
                    ++q;
                    if (M.flags & 2) break;
                }
                if (failed) break;
                mma_commit(smem_u32(&tfull_bar[buf]));
            }
            // every MMA issued by this thread has completed once this commit arrives
            mma_commit(smem_u32(&drain_bar));
            if (!mbar_wait(smem_u32(&drain_bar), 0)) failed = true;
        }
    } else {
        // ---------------- epilogue ----------------
        uint32_t tc = 0;
        for (int t = blockIdx.x; t < total && !failed; t += gridDim.x, ++tc) {
            const uint32_t buf = tc & 1u, use = tc >> 1;
            int ok = 1;
            if (lane == 0) ok = mbar_wait(smem_u32(&tfull_bar[buf]), use & 1u) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);  // warp-uniform (tcgen05.ld is warp-collective)
            if (!ok) { failed = true; break; }
            __syncwarp();
            tc_fence_after();
            const int tix = t / nvec, v = t % nvec;
            const Tile T = tiles[tix];
            const int nst = tile_stages(T, segs);
            epilogue_tile<NSPLIT>(T, v, nst, tmem + buf * TMEM_COLS, warp, lane, B, smem_u32(&tempty_bar[buf]));
        }
    }
    if (failed) {
        fail_s = 1;
        atomicExch(B.err, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(2 * TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// TMA-staged kernel
// ---------------------------------------------------------------------------

__device__ __forceinline__ void mbar_arrive_tx(uint32_t addr, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(addr), "r"(bytes) : "memory");
}
// 64 x 64 box of a 4-D tensor map into shared memory, completion on an mbarrier
__device__ __forceinline__ void tma_load4(uint32_t dst, const CUtensorMap* map, int x, int y, int z, int w,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
        : "memory");
}


// One 128 x 64 operand piece as (up to) two 64-row boxes.  K-major (mn = 0):
// rows r0.. of the map at x = k0; MN-major (mn = 1): columns r0.. of the map
// at rows k0..  Shared layout: K-major rows at 128 B (8-row groups 1 KB
// apart); MN-major 64-element halves 8 KB apart, 8-row K groups 1 KB apart.
// With halves = 1 the second half is not loaded (the block ends within the
// first 64 rows / columns; the MMA reads don't-care data there, which only
// reaches output rows / columns the epilogue drops).
__device__ __forceinline__ void tma_piece(uint32_t dst, const CUtensorMap* map, int mn, int r0, int k0, int z, int w,
                                          uint32_t bar, int halves) {
    if (!mn) {
        tma_load4(dst, map, k0, r0, z, w, bar);
        if (halves == 2) tma_load4(dst + 8192, map, k0, r0 + 64, z, w, bar);
    } else {
        tma_load4(dst, map, r0, k0, z, w, bar);
        if (halves == 2) tma_load4(dst + 8192, map, r0 + 64, k0, z, w, bar);
    }
}

// Roles: warps 0-3 epilogue (as in tc_seg_gemm_kernel), warp 4 lane 0 TMA
// producer, warp 5 lane 0 MMA issuer.
constexpr int THREADS3 = (kEpiWarps + 2) * 32;

template <int NSPLIT>
struct Cfg3 {
    static constexpr int STAGES = (NSPLIT == 1) ? 6 : (NSPLIT == 2 ? 3 : 2);
    static constexpr int STAGE_BYTES = 2 * NSPLIT * PIECE_BYTES;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
};

// stage record of the TMA kernel
struct StageMeta3 {
    uint8_t a_mn, b_mn, neg, flags;  // flags: 1 first stage of a tile, 2 last, 4 no MMA (empty tile)
    uint8_t k16, n16, pad[2];        // 16-deep K steps holding data; MMA N / 16
};

__device__ __forceinline__ uint32_t idesc_n(int a_mn, int b_mn, int neg, int n) { return idesc_mn(a_mn, b_mn, neg, n, TM); }

template <int NSPLIT>
__global__ void __launch_bounds__(THREADS3, 1)
    tc_tma_kernel(const Tile* __restrict__ tiles, int ntiles, int nvec, const TSeg* __restrict__ segs,
                  const CUtensorMap* __restrict__ maps, TcBufs B) {
    using C = Cfg3<NSPLIT>;
    constexpr int S = C::STAGES;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[S], empty_bar[S], tfull_bar[2], tempty_bar[2], drain_bar;
    __shared__ StageMeta3 meta[S];
    __shared__ uint32_t tmem_base_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_base_s)),
                     "r"(2 * TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&tfull_bar[b]), 1);
            mbar_init(smem_u32(&tempty_bar[b]), kEpiWarps);
        }
        mbar_init(smem_u32(&drain_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;
    const int total = ntiles * nvec;
    bool failed = false;

    if (warp == kEpiWarps) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            uint32_t q = 0;
            for (int t = blockIdx.x; t < total && !failed; t += gridDim.x) {
                const int v = t % nvec;
                const Tile T = tiles[t / nvec];
                const int nst = T.nst;
                // a second 64-row (or 64-column) half only when the block extends past the first
                const int ncol = min(T.tn, T.n - T.n0);  // columns of this tile
                const int nA = (T.m - T.m0 > 64) ? 2 : 1, nB = (ncol > 64) ? 2 : 1;
                const int n16 = (ncol + 15) / 16;
                if (nst == 0) {
                    if (q >= (uint32_t)S && !mbar_wait(smem_u32(&empty_bar[q % S]), ((q / S) - 1) & 1u)) {
                        failed = true;
                        break;
                    }
                    meta[q % S] = StageMeta3{0, 0, 0, 1 | 2 | 4, 0, 0, {0, 0}};
                    mbar_arrive(smem_u32(&full_bar[q % S]));
                    ++q;
                    continue;
                }
                int done = 0;
                for (int s = T.seg_beg; s < T.seg_end && !failed; ++s) {
                    const TSeg Sg = segs[s];
                    const int a_mn = Sg.a_tr ? 1 : 0, b_mn = Sg.b_tr ? 0 : 1;
                    const int aw = Sg.a_pv ? v : 0, bw = Sg.b_pv ? v : 0;
                    const CUtensorMap* am = maps + 3 * Sg.a_map;
                    const CUtensorMap* bm = maps + 3 * Sg.b_map;
                    const uint32_t bytes = (uint32_t)NSPLIT * 128u * (uint32_t)(nA * Sg.a_br + nB * Sg.b_br);
                    for (int k0 = 0; k0 < Sg.k; k0 += TK) {
                        const uint32_t slot = q % S;
                        if (q >= (uint32_t)S && !mbar_wait(smem_u32(&empty_bar[slot]), ((q / S) - 1) & 1u)) {
                            failed = true;
                            break;
                        }
                        const int kv = min(TK, Sg.k - k0);
                        meta[slot] = StageMeta3{(uint8_t)a_mn, (uint8_t)b_mn, (uint8_t)(Sg.sign < 0.f ? 1 : 0),
                                                (uint8_t)((done == 0 ? 1 : 0) | (done == nst - 1 ? 2 : 0)),
                                                (uint8_t)((kv + 15) / 16), (uint8_t)n16, {0, 0}};
                        const uint32_t bar = smem_u32(&full_bar[slot]);
                        mbar_arrive_tx(bar, bytes);
                        const uint32_t sa = sbase + slot * C::STAGE_BYTES;
                        const uint32_t sb = sa + NSPLIT * PIECE_BYTES;
#pragma unroll
                        for (int pc = 0; pc < NSPLIT; ++pc) {
                            tma_piece(sa + pc * PIECE_BYTES, am + pc, a_mn, T.m0, k0, Sg.a_z, aw, bar, nA);
                            tma_piece(sb + pc * PIECE_BYTES, bm + pc, b_mn, T.n0, k0, Sg.b_z, bw, bar, nB);
                        }
                        ++q;
                        ++done;
                    }
                }
            }
        }
    } else if (warp == kEpiWarps + 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            uint32_t q = 0, tc = 0;
            for (int t = blockIdx.x; t < total && !failed; t += gridDim.x, ++tc) {
                const uint32_t buf = tc & 1u, use = tc >> 1;
                if (use > 0 && !mbar_wait(smem_u32(&tempty_bar[buf]), (use - 1) & 1u)) {
                    failed = true;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem + buf * TMEM_COLS;
                for (;;) {
                    const uint32_t slot = q % S;
                    if (!mbar_wait(smem_u32(&full_bar[slot]), (q / S) & 1u)) {
                        failed = true;
                        break;
                    }
                    tc_fence_after();
                    const StageMeta3 M = meta[slot];
                    if (!(M.flags & 4)) {
                        const uint32_t sa = sbase + slot * C::STAGE_BYTES;
                        const uint32_t sb = sa + NSPLIT * PIECE_BYTES;
                        const uint32_t id = idesc_n(M.a_mn, M.b_mn, M.neg, 16 * M.n16);
                        for (int kk = 0; kk < M.k16; ++kk) {
#pragma unroll
                            for (int pr = 0; pr < Prods<NSPLIT>::N; ++pr) {
                                const int pa = prod_a(pr), pb = prod_b(pr);
                                const uint32_t a_s = sa + pa * PIECE_BYTES;
                                const uint32_t b_s = sb + pb * PIECE_BYTES;
                                const uint64_t ad =
                                    M.a_mn ? sdesc(a_s + kk * 2048, 8192, 1024) : sdesc(a_s + kk * 32, 16, 1024);
                                const uint64_t bd =
                                    M.b_mn ? sdesc(b_s + kk * 2048, 8192, 1024) : sdesc(b_s + kk * 32, 16, 1024);
                                const uint32_t acc = ((M.flags & 1) && kk == 0 && pr == 0) ? 0u : 1u;
                                mma_bf16(dt, ad, bd, id, acc);
                            }
                        }
                    }
                    mma_commit(smem_u32(&empty_bar[slot]));
                    ++q;
                    if (M.flags & 2) break;
                }
                if (failed) break;
                mma_commit(smem_u32(&tfull_bar[buf]));
            }
            mma_commit(smem_u32(&drain_bar));
            if (!mbar_wait(smem_u32(&drain_bar), 0)) failed = true;
        }
    } else {
        // ---------------- epilogue ----------------
        uint32_t tc = 0;
        Tile Tn{};
        if (blockIdx.x < total) Tn = tiles[blockIdx.x / nvec];
        for (int t = blockIdx.x; t < total && !failed; t += gridDim.x, ++tc) {
            const uint32_t buf = tc & 1u, use = tc >> 1;
            const Tile T = Tn;  // fetched one tile ahead, while the MMAs of this one run
            if (t + (int)gridDim.x < total) Tn = tiles[(t + gridDim.x) / nvec];
            int ok = 1;
            if (lane == 0) ok = mbar_wait(smem_u32(&tfull_bar[buf]), use & 1u) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);  // warp-uniform (tcgen05.ld is warp-collective)
            if (!ok) {
                failed = true;
                break;
            }
            __syncwarp();
            tc_fence_after();
            epilogue_tile<NSPLIT>(T, t % nvec, T.nst, tmem + buf * TMEM_COLS, warp, lane, B,
                                  smem_u32(&tempty_bar[buf]));
        }
    }
    if (failed) atomicExch(B.err, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(2 * TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// conversions
// ---------------------------------------------------------------------------

// x -> hi (+ lo (+ lo2)): each piece is the bf16 rounding of what the previous ones leave
__device__ __forceinline__ void split3(double xd, __nv_bfloat16* hi, __nv_bfloat16* lo, __nv_bfloat16* lo2,
                                      int64_t i) {
    const __nv_bfloat16 h = __float2bfloat16_rn((float)xd);
    hi[i] = h;
    if (lo) {
        const double r = xd - (double)__bfloat162float(h);
        const __nv_bfloat16 l = __float2bfloat16_rn((float)r);
        lo[i] = l;
        if (lo2) lo2[i] = __float2bfloat16_rn((float)(r - (double)__bfloat162float(l)));
    }
}

__global__ void split_f64_kernel(const double* __restrict__ src, int64_t rows, int n, int64_t lds,
                                 __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int64_t ldd,
                                 __nv_bfloat16* __restrict__ lo2) {
    const int64_t tot = rows * ldd;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / ldd, c = i % ldd;
        split3((c < n) ? src[r * lds + c] : 0.0, hi, lo, lo2, i);
    }
}

__global__ void split_f64_flat_kernel(const double* __restrict__ src, int64_t n, __nv_bfloat16* __restrict__ hi,
                                      __nv_bfloat16* __restrict__ lo, __nv_bfloat16* __restrict__ lo2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        split3(src[i], hi, lo, lo2, i);
}

__global__ void split_f32_kernel(const float* __restrict__ src, int64_t n, __nv_bfloat16* __restrict__ hi,
                                 __nv_bfloat16* __restrict__ lo, __nv_bfloat16* __restrict__ lo2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        split3((double)src[i], hi, lo, lo2, i);
}

__global__ void split_blocks_kernel(const double* __restrict__ src, const SplitJob* __restrict__ jobs,
                                    __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                    __nv_bfloat16* __restrict__ lo2) {
    const SplitJob J = jobs[blockIdx.x];
    const int64_t tot = (int64_t)J.rows * J.ld_dst;
    for (int64_t i = threadIdx.x; i < tot; i += blockDim.x) {
        const int r = (int)(i / J.ld_dst), c = (int)(i % J.ld_dst);
        split3((c < J.cols) ? src[J.src_off + (int64_t)r * J.ld_src + c] : 0.0, hi, lo, lo2, J.dst_off + i);
    }
}

int grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

int tc_num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

void launch_seg_gemm_tc(const WorkList& w, const TcBufs& b, int nvec, int nsplit, cudaStream_t st) {
    if (w.tiles.empty()) return;
    const int64_t total = (int64_t)w.tiles.size() * nvec;
    DMRG_REQUIRE(total < (1LL << 31), DMRG_EINVAL, "tensor-core work list too large");
    DMRG_CHECK_CUDA(cudaMemsetAsync(b.counter, 0, sizeof(int), st));
    const int grid = (int)std::min<int64_t>(total, tc_num_sms());
    if (nsplit == 3) {
        static bool attr = false;
        if (!attr) {
            DMRG_CHECK_CUDA(cudaFuncSetAttribute(tc_seg_gemm_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 Cfg2<3>::SMEM));
            attr = true;
        }
        tc_seg_gemm_kernel<3><<<grid, THREADS2, Cfg2<3>::SMEM, st>>>(w.d_tiles, (int)w.tiles.size(), nvec, w.d_segs, b);
    } else if (nsplit == 2) {
        static bool attr = false;
        if (!attr) {
            DMRG_CHECK_CUDA(cudaFuncSetAttribute(tc_seg_gemm_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 Cfg2<2>::SMEM));
            attr = true;
        }
        tc_seg_gemm_kernel<2><<<grid, THREADS2, Cfg2<2>::SMEM, st>>>(w.d_tiles, (int)w.tiles.size(), nvec, w.d_segs, b);
    } else {
        static bool attr = false;
        if (!attr) {
            DMRG_CHECK_CUDA(cudaFuncSetAttribute(tc_seg_gemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 Cfg2<1>::SMEM));
            attr = true;
        }
        tc_seg_gemm_kernel<1><<<grid, THREADS2, Cfg2<1>::SMEM, st>>>(w.d_tiles, (int)w.tiles.size(), nvec, w.d_segs, b);
    }
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// TMA work lists and tensor maps (host)
// ---------------------------------------------------------------------------

void TmaWorkList::add_block(int64_t c_off, int c_buf, int m, int n, int ldc, const std::vector<TSeg>& s, uint8_t mode,
                            int64_t kchunk, float alpha, int tn) {
    if (m <= 0 || n <= 0) return;
    DMRG_REQUIRE(tn == 64 || tn == TN, DMRG_EINVAL, "tile width must be 64 or 128");
    std::vector<std::pair<int, int>> chunks;
    const bool atomic = (mode == TC_ATOMIC_F64 || mode == TC_ATOMIC_F32);
    if (atomic && kchunk > 0) {
        int beg = 0;
        int64_t acc = 0;
        for (int i = 0; i < (int)s.size(); ++i) {
            if (acc > 0 && acc + s[i].k > kchunk) {
                chunks.push_back({beg, i});
                beg = i;
                acc = 0;
            }
            acc += s[i].k;
        }
        chunks.push_back({beg, (int)s.size()});
    } else {
        chunks.push_back({0, (int)s.size()});
    }
    for (auto& ch : chunks) {
        const int sb = (int)segs.size();
        int64_t nst = 0;
        for (int i = ch.first; i < ch.second; ++i) {
            segs.push_back(s[i]);
            nst += (s[i].k + TK - 1) / TK;
        }
        DMRG_REQUIRE(nst < 65536, DMRG_EINVAL, "tile with too many K stages (use a K-chunk)");
        const int se = (int)segs.size();
        for (int m0 = 0; m0 < m; m0 += TM)
            for (int n0 = 0; n0 < n; n0 += tn) {
                Tile t{};
                t.tn = tn;
                t.alpha = alpha;
                t.c_off = c_off;
                t.ldc = ldc;
                t.m = m;
                t.n = n;
                t.m0 = m0;
                t.n0 = n0;
                t.seg_beg = sb;
                t.seg_end = se;
                t.c_buf = (uint8_t)c_buf;
                t.mode = mode;
                t.nst = (uint16_t)nst;
                tiles.push_back(t);
            }
    }
}

void TmaWorkList::order_tiles() {
    // longest tiles first: CTAs take tiles round-robin, so the short ones fill
    // in at the end of the launch instead of a few long ones trailing.  A
    // stable counting sort on the stage count (< 65536): two linear passes
    // instead of an n log n sort of millions of records on every bond
    if (tiles.size() > 1) {
        int maxn = 0;
        for (const Tile& t : tiles) maxn = std::max(maxn, (int)t.nst);
        std::vector<size_t> pos((size_t)maxn + 2, 0);
        for (const Tile& t : tiles) ++pos[(size_t)(maxn - t.nst) + 1];
        for (size_t i = 1; i < pos.size(); ++i) pos[i] += pos[i - 1];
        std::vector<Tile> sorted(tiles.size());
        for (const Tile& t : tiles) sorted[pos[(size_t)(maxn - t.nst)]++] = t;
        tiles.swap(sorted);
    }
}

void TmaWorkList::upload(cudaStream_t st) {
    if (tiles.size() > cap_tiles) {
        if (d_tiles) cudaFree(d_tiles);
        cap_tiles = tiles.size() + 16;
        DMRG_CHECK_CUDA(cudaMalloc(&d_tiles, cap_tiles * sizeof(Tile)));
    }
    if (segs.size() > cap_segs) {
        if (d_segs) cudaFree(d_segs);
        cap_segs = segs.size() + 16;
        DMRG_CHECK_CUDA(cudaMalloc(&d_segs, cap_segs * sizeof(TSeg)));
    }
    if (!tiles.empty())
        DMRG_CHECK_CUDA(cudaMemcpyAsync(d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, st));
    if (!segs.empty())
        DMRG_CHECK_CUDA(cudaMemcpyAsync(d_segs, segs.data(), segs.size() * sizeof(TSeg), cudaMemcpyHostToDevice, st));
}

void TmaWorkList::release() {
    if (d_tiles) cudaFree(d_tiles);
    if (d_segs) cudaFree(d_segs);
    d_tiles = nullptr;
    d_segs = nullptr;
    cap_tiles = cap_segs = 0;
}

int MapTable::get(const MapKey& k) {
    auto it = index.find(k);
    if (it != index.end()) return it->second;
    DMRG_REQUIRE(k.cols >= 1 && k.rows >= 1 && k.nz >= 1 && k.nv >= 1, DMRG_EINVAL, "empty tensor-map extent");
    DMRG_REQUIRE(k.off % 8 == 0 && k.ld % 8 == 0 && k.zstride % 8 == 0 && k.vstride % 8 == 0, DMRG_EINVAL,
                 "tensor-map operand not 16-byte aligned");
    DMRG_REQUIRE(k.ld >= k.cols && k.zstride >= k.rows * k.ld && k.vstride >= k.nz * k.zstride, DMRG_EINVAL,
                 "tensor-map strides overlap");
    const int i = (int)keys.size();
    keys.push_back(k);
    index[k] = i;
    return i;
}

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        DMRG_CHECK_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        DMRG_REQUIRE(q == cudaDriverEntryPointSuccess && p, DMRG_ECUDA, "cuTensorMapEncodeTiled unavailable");
        fn = (EncodeTiledFn)p;
    }
    return fn;
}
}  // namespace

void MapTable::encode_upload(const TcBufs& tb, int nsplit, cudaStream_t st) {
    const size_t n = 3 * keys.size();
    std::vector<CUtensorMap> h(std::max<size_t>(n, 1));
    EncodeTiledFn fn = encode_fn();
    for (size_t i = 0; i < keys.size(); ++i) {
        const MapKey& k = keys[i];
        for (int pc = 0; pc < 3; ++pc) {
            const __nv_bfloat16* base =
                pc == 0 ? tb.hi[k.buf] : (pc == 1 ? tb.lo[k.buf] : (tb.lo[k.buf] ? tb.lo[k.buf] + tb.pstride[k.buf] : nullptr));
            if (pc >= nsplit || !base) {  // unused piece: a copy of the hi map
                h[3 * i + pc] = h[3 * i];
                continue;
            }
            DMRG_REQUIRE(base != nullptr, DMRG_EINVAL, "tensor map over an unset buffer");
            const cuuint64_t dims[4] = {(cuuint64_t)k.cols, (cuuint64_t)k.rows, (cuuint64_t)k.nz, (cuuint64_t)k.nv};
            const cuuint64_t strides[3] = {(cuuint64_t)k.ld * 2, (cuuint64_t)k.zstride * 2, (cuuint64_t)k.vstride * 2};
            const cuuint32_t box[4] = {64, (cuuint32_t)box_rows(k.rows), 1, 1};
            const cuuint32_t estr[4] = {1, 1, 1, 1};
            const CUresult r = fn(&h[3 * i + pc], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)(base + k.off), dims,
                                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            DMRG_REQUIRE(r == CUDA_SUCCESS, DMRG_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
        }
    }
    if (n > cap) {
        if (d_maps) cudaFree(d_maps);
        cap = n + 64;
        DMRG_CHECK_CUDA(cudaMalloc(&d_maps, cap * sizeof(CUtensorMap)));
    }
    if (n > 0) DMRG_CHECK_CUDA(cudaMemcpyAsync(d_maps, h.data(), n * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    for (int b = 0; b < kMaxBufs; ++b) {
        enc_ptr[b][0] = tb.hi[b];
        enc_ptr[b][1] = tb.lo[b];
        enc_ptr[b][2] = tb.lo[b] ? tb.lo[b] + tb.pstride[b] : nullptr;
    }
}

bool MapTable::stale(const TcBufs& tb) const {
    if (!d_maps) return true;
    for (const MapKey& k : keys)
        if (enc_ptr[k.buf][0] != tb.hi[k.buf] || enc_ptr[k.buf][1] != tb.lo[k.buf] ||
            enc_ptr[k.buf][2] != (tb.lo[k.buf] ? tb.lo[k.buf] + tb.pstride[k.buf] : nullptr))
            return true;
    return false;
}

void MapTable::release() {
    if (d_maps) cudaFree(d_maps);
    d_maps = nullptr;
    cap = 0;
    clear();
}

void tc_prepare(int nsplit) {
    static bool done[4] = {false, false, false, false};
    if (nsplit < 1 || nsplit > 3 || done[nsplit]) return;
    if (nsplit == 1) {
        DMRG_CHECK_CUDA(cudaFuncSetAttribute(tc_tma_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg3<1>::SMEM));
    } else if (nsplit == 2) {
        DMRG_CHECK_CUDA(cudaFuncSetAttribute(tc_tma_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg3<2>::SMEM));
    } else {
        DMRG_CHECK_CUDA(cudaFuncSetAttribute(tc_tma_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg3<3>::SMEM));
    }
    done[nsplit] = true;
}

void launch_seg_gemm_tma(const TmaWorkList& w, const MapTable& maps, const TcBufs& b, int nvec, int nsplit,
                         cudaStream_t st) {
    tc_prepare(nsplit);
    if (w.tiles.empty()) return;
    const int64_t total = (int64_t)w.tiles.size() * nvec;
    DMRG_REQUIRE(total < (1LL << 31), DMRG_EINVAL, "tensor-core work list too large");
    DMRG_REQUIRE(maps.d_maps != nullptr, DMRG_EINVAL, "tensor maps not uploaded");
    const int grid = (int)std::min<int64_t>(total, tc_num_sms());
    if (nsplit == 3) {
        tc_tma_kernel<3><<<grid, THREADS3, Cfg3<3>::SMEM, st>>>(w.d_tiles, (int)w.tiles.size(), nvec, w.d_segs,
                                                        maps.d_maps, b);
    } else if (nsplit == 2) {
        tc_tma_kernel<2><<<grid, THREADS3, Cfg3<2>::SMEM, st>>>(w.d_tiles, (int)w.tiles.size(), nvec, w.d_segs,
                                                               maps.d_maps, b);
    } else {
        tc_tma_kernel<1><<<grid, THREADS3, Cfg3<1>::SMEM, st>>>(w.d_tiles, (int)w.tiles.size(), nvec, w.d_segs,
                                                               maps.d_maps, b);
    }
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

void dev_split_f64(const double* src, int64_t rows, int n, int64_t ld_src, __nv_bfloat16* hi, __nv_bfloat16* lo,
                   int64_t ld_dst, cudaStream_t st, __nv_bfloat16* lo2) {
    if (rows <= 0) return;
    split_f64_kernel<<<grid_for(rows * ld_dst), 256, 0, st>>>(src, rows, n, ld_src, hi, lo, ld_dst, lo2);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

void dev_split_f64_flat(const double* src, int64_t n, __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t st,
                        __nv_bfloat16* lo2) {
    if (n <= 0) return;
    split_f64_flat_kernel<<<grid_for(n), 256, 0, st>>>(src, n, hi, lo, lo2);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

void dev_split_f32(const float* src, int64_t n, __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t st,
                   __nv_bfloat16* lo2) {
    if (n <= 0) return;
    split_f32_kernel<<<grid_for(n), 256, 0, st>>>(src, n, hi, lo, lo2);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

void dev_split_blocks(const double* src, const SplitJob* d_jobs, int njobs, __nv_bfloat16* hi, __nv_bfloat16* lo,
                      cudaStream_t st, __nv_bfloat16* lo2) {
    if (njobs <= 0) return;
    split_blocks_kernel<<<njobs, 256, 0, st>>>(src, d_jobs, hi, lo, lo2);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

}  // namespace dmrg

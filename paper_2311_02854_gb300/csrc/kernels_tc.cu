// Tensor-core segmented grouped GEMM for sm_103a (5th-generation tensor cores):
// operands staged in shared memory (128B-swizzled canonical layouts, K-major
// or MN-major), tcgen05.mma kind::f16 with bf16 inputs and FP32 accumulation
// in tensor memory, completion tracked by mbarriers, persistent CTAs pulling
// tiles from a counter.  One output tile (128 x 128) accumulates the whole
// list of K-segments of its block (the term sum of Eq. sigmablk happens in
// the accumulator).  bf16 "pieces": an operand x is held as hi + lo; with
// nsplit = 2 each product runs as hi*hi + hi*lo + lo*hi.
#include <cuda_bf16.h>

#include <algorithm>

#include "tc.h"

namespace dmrg {
namespace {

constexpr int TM = 128, TN = 128, TK = 64, THREADS = 128;
constexpr int PIECE_BYTES = TM * TK * 2;  // one 128 x 64 bf16 operand tile
constexpr uint32_t TMEM_COLS = 128;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // bounded waits: 2 s

template <int NSPLIT>
struct Cfg {
    static constexpr int STAGES = (NSPLIT == 1) ? 4 : 3;
    static constexpr int STAGE_BYTES = 2 * NSPLIT * PIECE_BYTES;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait until the phase with the given parity has completed; false on timeout.
__device__ bool mbar_wait(uint32_t addr, uint32_t parity) {
    if (mbar_try(addr, parity)) return true;
    const uint64_t t0 = gtimer();
    while (!mbar_try(addr, parity)) {
        if (gtimer() - t0 > kWaitLimitNs) return false;
    }
    return true;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// smem matrix descriptor (tcgen05): start >> 4, LBO >> 4, SBO >> 4, version 1, 128B swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// instruction descriptor, kind::f16: D f32, A/B bf16, majors, negate A, N, M
__device__ __forceinline__ uint32_t idesc(int a_mn, int b_mn, int neg) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)neg << 13) | ((uint32_t)a_mn << 15) |
           ((uint32_t)b_mn << 16) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(id), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// Stage one 128 x 64 tile of an operand into shared memory.
// Element (r, k) of the operand lives at base[r*ld + k] (mn = 0: K-major) or
// base[k*ld + r] (mn = 1: MN-major); valid for r < R, k < K (zero-filled outside).
__device__ __forceinline__ void load_tile(uint32_t sdst, const __nv_bfloat16* base, int ld, int mn, int r0, int R,
                                          int k0, int K, int tid) {
    if (!mn) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int idx = tid + i * THREADS;
            const int r = idx >> 3, c = idx & 7;
            const int kk = k0 + c * 8;
            int valid = 0;
            const __nv_bfloat16* src = base;
            if (r0 + r < R && kk < K) {
                valid = min(8, K - kk);
                src = base + (int64_t)(r0 + r) * ld + kk;
            }
            const uint32_t dst = sdst + (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
            cp_async16(dst, src, valid * 2);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int idx = tid + i * THREADS;
            const int kr = idx >> 4, c = idx & 15;
            const int rr = r0 + c * 8;
            int valid = 0;
            const __nv_bfloat16* src = base;
            if (k0 + kr < K && rr < R) {
                valid = min(8, R - rr);
                src = base + (int64_t)(k0 + kr) * ld + rr;
            }
            const uint32_t dst =
                sdst + (uint32_t)((((kr >> 3) * 2 + (c >> 3)) * 1024) + (kr & 7) * 128 + (((c & 7) ^ (kr & 7)) << 4));
            cp_async16(dst, src, valid * 2);
        }
    }
}

template <int NSPLIT>
__global__ void __launch_bounds__(THREADS, 1)
    tc_seg_gemm_kernel(const Tile* __restrict__ tiles, int ntiles, int nvec, const Seg* __restrict__ segs, TcBufs B) {
    using C = Cfg<NSPLIT>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bars[C::STAGES];
    __shared__ uint32_t tmem_base_s;
    __shared__ int tile_s;
    __shared__ int stage_mn[C::STAGES][3];  // a_mn, b_mn, neg of the stage held in a slot
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_base_s)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < C::STAGES; ++s) mbar_init(smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    const int total = ntiles * nvec;
    uint32_t g = 0;  // stages issued by this CTA (slot = g % STAGES)
    bool failed = false;
    for (;;) {
        if (tid == 0) tile_s = atomicAdd(B.counter, 1);
        __syncthreads();
        const int idx = tile_s;
        if (idx >= total) break;
        const int tix = idx % ntiles, v = idx / ntiles;
        const Tile T = tiles[tix];
        int nst = 0;
        for (int s = T.seg_beg; s < T.seg_end; ++s) nst += (segs[s].k + TK - 1) / TK;

        if (nst > 0) {
            int ls = T.seg_beg, lk = 0;  // load cursor
            while (ls < T.seg_end && lk >= segs[ls].k) { ++ls; lk = 0; }
            int ms = ls, mk = 0;         // mma cursor
            auto issue_load = [&](uint32_t q) -> bool {
                const uint32_t slot = q % C::STAGES;
                if (q >= (uint32_t)C::STAGES) {
                    if (!mbar_wait(smem_u32(&bars[slot]), ((q - C::STAGES) / C::STAGES) & 1u)) return false;
                }
                const Seg S = segs[ls];
                const int a_mn = S.a_tr ? 1 : 0;
                const int b_mn = S.b_tr ? 0 : 1;
                const uint32_t sa = sbase + slot * C::STAGE_BYTES;
                const uint32_t sb = sa + NSPLIT * PIECE_BYTES;
                const int64_t ao = S.a_off + (int64_t)v * B.vstride[S.a_buf];
                const int64_t bo = S.b_off + (int64_t)v * B.vstride[S.b_buf];
                load_tile(sa, B.hi[S.a_buf] + ao, S.lda, a_mn, T.m0, T.m, lk, S.k, tid);
                load_tile(sb, B.hi[S.b_buf] + bo, S.ldb, b_mn, T.n0, T.n, lk, S.k, tid);
                if (NSPLIT == 2) {
                    load_tile(sa + PIECE_BYTES, B.lo[S.a_buf] + ao, S.lda, a_mn, T.m0, T.m, lk, S.k, tid);
                    load_tile(sb + PIECE_BYTES, B.lo[S.b_buf] + bo, S.ldb, b_mn, T.n0, T.n, lk, S.k, tid);
                }
                if (tid == 0) {
                    stage_mn[slot][0] = a_mn;
                    stage_mn[slot][1] = b_mn;
                    stage_mn[slot][2] = S.alpha < 0.0 ? 1 : 0;
                }
                cp_async_commit();
                lk += TK;
                while (ls < T.seg_end && lk >= segs[ls].k) { ++ls; lk = 0; }
                return true;
            };
            bool ok = issue_load(g);
            for (int t = 0; t < nst && ok; ++t) {
                if (t + 1 < nst) {
                    ok = issue_load(g + t + 1);
                    cp_async_wait1();
                } else {
                    cp_async_wait0();
                }
                fence_proxy_async();
                if (__syncthreads_or(!ok)) {
                    ok = false;
                    break;
                }
                if (tid == 0) {
                    tc_fence_after();
                    const uint32_t slot = (g + t) % C::STAGES;
                    const uint32_t sa = sbase + slot * C::STAGE_BYTES;
                    const uint32_t sb = sa + NSPLIT * PIECE_BYTES;
                    const int a_mn = stage_mn[slot][0], b_mn = stage_mn[slot][1], neg = stage_mn[slot][2];
                    const uint32_t id = idesc(a_mn, b_mn, neg);
#pragma unroll
                    for (int kk = 0; kk < TK / 16; ++kk) {
#pragma unroll
                        for (int p = 0; p < (NSPLIT == 2 ? 3 : 1); ++p) {
                            const int pa = (p == 2) ? 1 : 0;  // products: hi*hi, hi*lo, lo*hi
                            const int pb = (p == 1) ? 1 : 0;
                            const uint32_t a_s = sa + pa * PIECE_BYTES;
                            const uint32_t b_s = sb + pb * PIECE_BYTES;
                            const uint64_t ad = a_mn ? sdesc(a_s + kk * 4096, 1024, 2048) : sdesc(a_s + kk * 32, 16, 1024);
                            const uint64_t bd = b_mn ? sdesc(b_s + kk * 4096, 1024, 2048) : sdesc(b_s + kk * 32, 16, 1024);
                            const uint32_t acc = (t == 0 && kk == 0 && p == 0) ? 0u : 1u;
                            mma_bf16(tmem, ad, bd, id, acc);
                        }
                    }
                    mma_commit(smem_u32(&bars[slot]));
                }
                mk += TK;
                while (ms < T.seg_end && mk >= segs[ms].k) { ++ms; mk = 0; }
            }
            if (!ok) {
                failed = true;
                g += nst;
                break;
            }
            g += nst;
            // all MMAs of the tile are complete once the last commit has arrived
            const uint32_t last = g - 1;
            const bool done = mbar_wait(smem_u32(&bars[last % C::STAGES]), (last / C::STAGES) & 1u);
            if (__syncthreads_or(!done)) {
                failed = true;
                break;
            }
            tc_fence_after();
        }

        // epilogue: TMEM lane = output row (warp w owns rows 32w..32w+31)
        const int row = warp * 32 + lane;
        const int r = T.m0 + row;
        const bool rok = r < T.m;
        const float alpha = T.alpha;
        for (int cg = 0; cg < TN / 32; ++cg) {
            uint32_t acc[32];
            if (nst > 0) {
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cg * 32), acc);
                tmem_wait_ld();
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[j] = 0u;
            }
            const int c0 = T.n0 + cg * 32;
            if (!rok || c0 >= T.n) continue;
            const int ncol = min(32, T.n - c0);
            const int64_t off = T.c_off + (int64_t)r * T.ldc + c0 + (int64_t)v * B.out_vstride[T.c_buf];
            if (T.mode == TC_ATOMIC_F64) {
                if (nst == 0) continue;
                double* o = (double*)B.out[T.c_buf] + off;
                for (int j = 0; j < ncol; ++j) atomicAdd(o + j, (double)alpha * (double)__uint_as_float(acc[j]));
            } else if (T.mode == TC_ATOMIC_F32) {
                if (nst == 0) continue;
                float* o = (float*)B.out[T.c_buf] + off;
                for (int j = 0; j < ncol; ++j) atomicAdd(o + j, alpha * __uint_as_float(acc[j]));
            } else if (T.mode == TC_STORE_F32) {
                float* o = (float*)B.out[T.c_buf] + off;
                for (int j = 0; j < ncol; ++j) o[j] = alpha * __uint_as_float(acc[j]);
            } else {  // TC_STORE_SPLIT: chunks of 8 (rows padded to multiples of 8)
                __nv_bfloat16* oh = (__nv_bfloat16*)B.out[T.c_buf] + off;
                __nv_bfloat16* ol = (__nv_bfloat16*)B.out_lo[T.c_buf] + off;
                for (int j0 = 0; j0 < ncol; j0 += 8) {
                    __align__(16) __nv_bfloat16 h8[8], l8[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float x = alpha * __uint_as_float(acc[j0 + j]);
                        const __nv_bfloat16 h = __float2bfloat16_rn(x);
                        h8[j] = h;
                        l8[j] = __float2bfloat16_rn(x - __bfloat162float(h));
                    }
                    *(uint4*)(oh + j0) = *(const uint4*)h8;
                    if (NSPLIT == 2) *(uint4*)(ol + j0) = *(const uint4*)l8;
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    if (failed && tid == 0) atomicExch(B.err, 1);
    // make sure no MMA is in flight before releasing tensor memory
    if (failed && g > 0) {
        const uint32_t last = g - 1;
        (void)mbar_wait(smem_u32(&bars[last % C::STAGES]), (last / C::STAGES) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// conversions
// ---------------------------------------------------------------------------

__global__ void split_f64_kernel(const double* __restrict__ src, int64_t rows, int n, int64_t lds,
                                 __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int64_t ldd) {
    const int64_t tot = rows * ldd;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / ldd, c = i % ldd;
        const float x = (c < n) ? (float)src[r * lds + c] : 0.0f;
        const double xd = (c < n) ? src[r * lds + c] : 0.0;
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi[i] = h;
        if (lo) lo[i] = __float2bfloat16_rn((float)(xd - (double)__bfloat162float(h)));
    }
}

__global__ void split_f32_kernel(const float* __restrict__ src, int64_t n, __nv_bfloat16* __restrict__ hi,
                                 __nv_bfloat16* __restrict__ lo) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = src[i];
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi[i] = h;
        if (lo) lo[i] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}

__global__ void split_blocks_kernel(const double* __restrict__ src, const SplitJob* __restrict__ jobs,
                                    __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
    const SplitJob J = jobs[blockIdx.x];
    const int64_t tot = (int64_t)J.rows * J.ld_dst;
    for (int64_t i = threadIdx.x; i < tot; i += blockDim.x) {
        const int r = (int)(i / J.ld_dst), c = (int)(i % J.ld_dst);
        const double xd = (c < J.cols) ? src[J.src_off + (int64_t)r * J.ld_src + c] : 0.0;
        const __nv_bfloat16 h = __float2bfloat16_rn((float)xd);
        hi[J.dst_off + i] = h;
        if (lo) lo[J.dst_off + i] = __float2bfloat16_rn((float)(xd - (double)__bfloat162float(h)));
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
    if (nsplit == 2) {
        static bool attr = false;
        if (!attr) {
            DMRG_CHECK_CUDA(cudaFuncSetAttribute(tc_seg_gemm_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 Cfg<2>::SMEM));
            attr = true;
        }
        tc_seg_gemm_kernel<2><<<grid, THREADS, Cfg<2>::SMEM, st>>>(w.d_tiles, (int)w.tiles.size(), nvec, w.d_segs, b);
    } else {
        static bool attr = false;
        if (!attr) {
            DMRG_CHECK_CUDA(cudaFuncSetAttribute(tc_seg_gemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 Cfg<1>::SMEM));
            attr = true;
        }
        tc_seg_gemm_kernel<1><<<grid, THREADS, Cfg<1>::SMEM, st>>>(w.d_tiles, (int)w.tiles.size(), nvec, w.d_segs, b);
    }
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

void dev_split_f64(const double* src, int64_t rows, int n, int64_t ld_src, __nv_bfloat16* hi, __nv_bfloat16* lo,
                   int64_t ld_dst, cudaStream_t st) {
    if (rows <= 0) return;
    split_f64_kernel<<<grid_for(rows * ld_dst), 256, 0, st>>>(src, rows, n, ld_src, hi, lo, ld_dst);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

void dev_split_f32(const float* src, int64_t n, __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t st) {
    if (n <= 0) return;
    split_f32_kernel<<<grid_for(n), 256, 0, st>>>(src, n, hi, lo);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

void dev_split_blocks(const double* src, const SplitJob* d_jobs, int njobs, __nv_bfloat16* hi, __nv_bfloat16* lo,
                      cudaStream_t st) {
    if (njobs <= 0) return;
    split_blocks_kernel<<<njobs, 256, 0, st>>>(src, d_jobs, hi, lo);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

}  // namespace dmrg

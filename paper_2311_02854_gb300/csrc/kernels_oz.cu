// FP64-accurate segmented grouped GEMM on the bf16 tensor cores of sm_103a.
//
// GB300 runs FP64 at ~1.2 TFLOP/s, so the products that must be FP64-accurate
// (the FP64 operator store, the residuals of the defect correction, FP64
// Rayleigh quotients) are emulated on the bf16 tensor cores by an error-free
// splitting of the operands (Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 59, 2012):
//
//  * every 32-deep K stage of a 128 x 64 output tile is converted by loader
//    warps: row r of A and column c of B get a power-of-two scale 2^E from the
//    largest magnitude in their 32 elements, the element is rounded to a
//    48-bit integer Q = round(|x| 2^(48-E)), and Q is cut into six 8-bit
//    slices q_0..q_5 (q_0 <= 256) stored as bf16 (exact: at most 9 significant
//    bits), so that x = sign * sum_i q_i 2^(E - 8(i+1)) up to 2^(E-49);
//  * the slice products with i + j = g <= 5 are issued as tcgen05.mma
//    (M = 128, N = 64, K = 16 per instruction) into one FP32 accumulator per
//    order g in tensor memory.  Every product is an integer below 2^16 and
//    each order's sum over the 32-deep stage stays below 2^24 for g <= 5, so
//    the accumulations are exact whatever the order of the additions;
//  * the epilogue warps read the six orders, combine them with the row and
//    column scales and the segment's alpha into a double-float (two FP32)
//    accumulator per element (FP32 arithmetic only: GB300's FP32 rate is ~64x
//    its FP64 rate), and at the end of the tile write or atomically add the
//    FP64 result.
//
// The work list is the FP64 engine's (Tile / Seg records over FP64 buffers of
// a BufTable), lowered with 128 x 64 tiles and uploaded longest first.
// Persistent CTAs, one per SM, walk (tile, vector) items with the vectors
// innermost, so the CTAs that run at the same time share their operator tiles
// in L2.  Slices are kept in 128B-swizzled rows 64 deep that hold two stages,
// so stage q+1 is converted into the other half while the tensor cores consume
// stage q.  Warps 0-7 epilogue (warp w: tile rows 32 (w % 4) .., columns
// 32 (w / 4) ..), warps 8-11 loaders (A rows one per thread, B columns two
// threads each), warp 12 lane 0 issues the MMAs.  Every wait is bounded; a
// timeout sets the device error word.
#include <cuda_bf16.h>

#include <algorithm>

#include "engine.h"
#include "ptx.h"

namespace dmrg {
namespace {

using namespace ptx;

constexpr int OTM = 128, OTN = 64, OTK = 32;   // tile rows, columns, stage depth
constexpr int ROWK = 64;                       // K of a swizzled slice row (two stages)
constexpr int NSL = 6;                         // slices per operand
constexpr int NORD = 6;                        // accumulated orders g = i + j = 0..5
constexpr int A_SLICE = OTM * ROWK * 2;        // 16 KB
constexpr int B_SLICE = OTN * ROWK * 2;        // 8 KB
constexpr int SLICE_BYTES = NSL * (A_SLICE + B_SLICE);
constexpr int EXP_SLOTS = 4;
constexpr uint32_t TMEM_COLS = 512;            // 6 orders x 64 columns, rounded to a power of two
// warps 0-7 epilogue (warp w: tile rows 32 (w % 4) .., columns 32 (w / 4) ..),
// warps 8-11 loaders, warp 12 lane 0 MMA issuer; 13 warps keep 4 per SM
// sub-partition, i.e. up to 128 registers per thread
constexpr int NEPI = 8;
constexpr int OZ_THREADS = (NEPI + 4 + 1) * 32;
constexpr int NLOAD = 128;
constexpr int EPI_COLS = OTN / 2;

// per-stage record shared by loaders (write) and epilogue (read)
struct OzStage {
    int32_t ea[OTM];   // row scales of A (exponent E: |x| < 2^E), -1000 for a zero row
    int32_t eb[OTN];   // column scales of B
    float ah, al;      // alpha as a double-float pair
    int32_t flags;     // 1 first stage of the tile, 2 last, 4 no MMA (tile without stages)
    int32_t pad;
};
// the low parts of the epilogue's double-float accumulators live in shared
// memory ([column][thread], conflict-free), the high parts in registers
constexpr int ACL_BYTES = NEPI * 32 * EPI_COLS * 4;
constexpr int OZ_SMEM = 1024 + SLICE_BYTES + EXP_SLOTS * (int)sizeof(OzStage) + ACL_BYTES;

// biased exponent field of a double from its high 32-bit word (0 for zero and subnormals)
__device__ __forceinline__ int exp_field_hi(int hi) { return (hi >> 20) & 0x7FF; }

// 48-bit integer magnitude of |x| 2^(48-E) (rounded half up), with E = ebias - 1023
__device__ __forceinline__ uint64_t q48(double x, int ebias) {
    const uint64_t bits = (uint64_t)__double_as_longlong(x);
    const int eb = (int)((bits >> 52) & 0x7FF);
    if (eb == 0) return 0;  // zero / subnormal: below every scale used here
    const uint64_t m = (bits & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const int sh = ebias + 4 - eb;  // right shift, >= 5
    if (sh >= 54) return 0;
    return (m + (1ull << (sh - 1))) >> sh;
}

// bf16 bit pattern of the integer q (0..256) with the given sign bit
__device__ __forceinline__ uint32_t bf16_of_int(uint32_t q, uint32_t sign) {
    const float f = __uint_as_float(0x4B000000u | q) - 8388608.0f;
    return (__float_as_uint(f) >> 16) | (sign << 15);
}

// Convert N values (read by ld(kk), kk = 0..N-1) into the six slices at
// dst + s * slice_bytes: row `row` of a 128B-swizzled K-major tile, 16-byte
// chunks cbase .. cbase + N/8 - 1 of the row.
template <int N, class Ld>
__device__ __forceinline__ void store_slices(const Ld& ld, int ebias, uint32_t dst, int slice_bytes, int row,
                                             int cbase) {
    const uint32_t rowoff = (uint32_t)((row >> 3) * 1024 + (row & 7) * 128);
#pragma unroll
    for (int cl = 0; cl < N / 8; ++cl) {
        uint32_t w[NSL][4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            uint32_t b16[2][NSL];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const double v = ld(cl * 8 + 2 * p + h);
                const uint32_t sign = (uint32_t)(__double2hiint(v) >> 31) & 1u;
                const uint64_t Q = q48(v, ebias);
                const uint32_t ql = (uint32_t)Q, qh = (uint32_t)(Q >> 32);
                b16[h][0] = bf16_of_int(qh >> 8, sign);
                b16[h][1] = bf16_of_int(qh & 255u, sign);
                b16[h][2] = bf16_of_int(ql >> 24, sign);
                b16[h][3] = bf16_of_int((ql >> 16) & 255u, sign);
                b16[h][4] = bf16_of_int((ql >> 8) & 255u, sign);
                b16[h][5] = bf16_of_int(ql & 255u, sign);
            }
#pragma unroll
            for (int s = 0; s < NSL; ++s) w[s][p] = b16[0][s] | (b16[1][s] << 16);
        }
        const int c = cbase + cl;
        const uint32_t off = rowoff + (uint32_t)(((c ^ (row & 7)) & 7) << 4);
#pragma unroll
        for (int s = 0; s < NSL; ++s)
            asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};\n" ::"r"(dst + s * slice_bytes + off), "r"(w[s][0]),
                         "r"(w[s][1]), "r"(w[s][2]), "r"(w[s][3])
                         : "memory");
    }
}

__device__ __forceinline__ void loaders_sync() { asm volatile("bar.sync 1, 128;\n" ::: "memory"); }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// exactly representable FP32 power of two 2^k (0 below the normal range)
__device__ __forceinline__ float pow2f(int k) {
    if (k < -126) return 0.0f;
    if (k > 127) k = 127;
    return __uint_as_float((uint32_t)(k + 127) << 23);
}

__device__ __forceinline__ int tile_nst(const Tile& T, const Seg* __restrict__ segs) {
    int nst = 0;
    for (int s = T.seg_beg; s < T.seg_end; ++s) nst += (segs[s].k + OTK - 1) / OTK;
    return nst;
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_gemm_kernel(const Tile* __restrict__ tiles, int ntiles, int nvec, const Seg* __restrict__ segs, BufTable bt,
                   int* err) {
    extern __shared__ uint8_t smem_raw[];
    // full[h]: loaders -> MMA (slices of K half h and the stage record written);
    // stage: MMA -> epilogue (stage record visible; arrived after the previous
    // accumulators were read); mma[h]: MMA completion -> loaders (half h free)
    // and epilogue (orders ready); free: epilogue -> MMA (accumulators read)
    __shared__ __align__(8) uint64_t full_bar[2], mma_bar[2], stage_bar, free_bar, drain_bar;
    __shared__ uint32_t tmem_base_s;
    __shared__ int32_t ebp[2][OTN];  // per-part column exponent fields of B (loaders)
    __shared__ int32_t load_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t sA = sbase, sB = sbase + NSL * A_SLICE;
    OzStage* stages = reinterpret_cast<OzStage*>(smem_raw + (sbase - smem_u32(smem_raw)) + SLICE_BYTES);
    float* acl_s = reinterpret_cast<float*>(stages + EXP_SLOTS);

    if (warp == 0) tmem_alloc(smem_u32(&tmem_base_s), TMEM_COLS);
    if (tid == 0) {
        for (int h = 0; h < 2; ++h) {
            mbar_init(smem_u32(&full_bar[h]), NLOAD);
            mbar_init(smem_u32(&mma_bar[h]), 1);
        }
        mbar_init(smem_u32(&stage_bar), 1);
        mbar_init(smem_u32(&free_bar), NEPI);
        mbar_init(smem_u32(&drain_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;
    const int total = ntiles * nvec;
    bool failed = false;

    if (warp >= NEPI && warp < NEPI + 4) {
        // ---------------- loaders / converters ----------------
        const int t = tid - NEPI * 32;
        uint32_t q = 0;
        // K half (q & 1) of the slices is free once the MMAs of stage q - 2
        // completed; one thread waits and the decision is shared, so the loaders
        // stay uniform
        auto begin = [&]() -> bool {
            if (t == 0)
                load_ok = (q < 2 || mbar_wait(smem_u32(&mma_bar[q & 1u]), ((q >> 1) - 1) & 1u)) ? 1 : 0;
            loaders_sync();
            const bool ok = load_ok != 0;
            loaders_sync();
            return ok;
        };
        for (int it = blockIdx.x; it < total && !failed; it += gridDim.x) {
            const Tile T = tiles[it / nvec];
            const int v = it % nvec;
            const int nst = tile_nst(T, segs);
            int done = 0;
            if (nst == 0) {
                if (!begin()) { failed = true; break; }
                OzStage& S = stages[q % EXP_SLOTS];
                if (t == 0) {
                    S.flags = 1 | 2 | 4;
                    S.ah = S.al = 0.f;
                }
                fence_proxy_async();
                mbar_arrive(smem_u32(&full_bar[q & 1u]));
                ++q;
                continue;
            }
            for (int s = T.seg_beg; s < T.seg_end && !failed; ++s) {
                const Seg Sg = segs[s];
                const double* A = bt.p[Sg.a_buf] + Sg.a_off + (int64_t)v * bt.vstride[Sg.a_buf];
                const double* B = bt.p[Sg.b_buf] + Sg.b_off + (int64_t)v * bt.vstride[Sg.b_buf];
                for (int k0 = 0; k0 < Sg.k; k0 += OTK) {
                    if (!begin()) { failed = true; break; }
                    OzStage& S = stages[q % EXP_SLOTS];
                    const int cbase = (int)(q & 1u) * (OTK / 8);
                    // A: thread t converts row m0 + t over k0 .. k0+31: the row's scale
                    // from the high words (32 loads in flight), then the values
                    {
                        const int gi = T.m0 + t;
                        const bool rv = gi < T.m;
                        const int kn = rv ? min(OTK, Sg.k - k0) : 0;
                        auto idx = [&](int kk) -> int64_t {
                            const int k = k0 + kk;
                            return Sg.a_tr ? (int64_t)k * Sg.lda + gi : (int64_t)gi * Sg.lda + k;
                        };
                        int emax = 0;
#pragma unroll
                        for (int kk = 0; kk < OTK; ++kk)
                            if (kk < kn) emax = max(emax, exp_field_hi(reinterpret_cast<const int*>(A + idx(kk))[1]));
                        const int ebias = emax + 1;  // |x| < 2^(ebias - 1023)
                        S.ea[t] = emax ? ebias - 1023 : -1000;
                        auto lda = [&](int kk) -> double { return kk < kn ? A[idx(kk)] : 0.0; };
                        store_slices<OTK>(lda, ebias, sA, A_SLICE, t, cbase);
                    }
                    // B: threads t and t + 64 convert column (t & 63), K parts of 16
                    {
                        const int c = t & 63, part = t >> 6;
                        const int gj = T.n0 + c;
                        const int kb = k0 + 16 * part;
                        const int kn = gj < T.n ? max(0, min(16, Sg.k - kb)) : 0;
                        auto idx = [&](int kk) -> int64_t {
                            const int k = kb + kk;
                            return Sg.b_tr ? (int64_t)gj * Sg.ldb + k : (int64_t)k * Sg.ldb + gj;
                        };
                        int emax = 0;
#pragma unroll
                        for (int kk = 0; kk < 16; ++kk)
                            if (kk < kn) emax = max(emax, exp_field_hi(reinterpret_cast<const int*>(B + idx(kk))[1]));
                        ebp[part][c] = emax;
                        loaders_sync();
                        emax = max(ebp[0][c], ebp[1][c]);
                        const int ebias = emax + 1;
                        if (part == 0) S.eb[c] = emax ? ebias - 1023 : -1000;
                        auto ldb = [&](int kk) -> double { return kk < kn ? B[idx(kk)] : 0.0; };
                        store_slices<16>(ldb, ebias, sB, B_SLICE, c, cbase + 2 * part);
                    }
                    if (t == 0) {
                        const float ah = (float)Sg.alpha;
                        S.ah = ah;
                        S.al = (float)(Sg.alpha - (double)ah);
                        S.flags = (done == 0 ? 1 : 0) | (done == nst - 1 ? 2 : 0);
                    }
                    fence_proxy_async();
                    mbar_arrive(smem_u32(&full_bar[q & 1u]));
                    ++q;
                    ++done;
                }
            }
        }
    } else if (warp == NEPI + 4) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            uint32_t q = 0;
            const uint32_t id = idesc_mn(0, 0, 0, OTN, OTM);
            for (int it = blockIdx.x; it < total && !failed; it += gridDim.x) {
                const Tile T = tiles[it / nvec];
                int nst = tile_nst(T, segs);
                if (nst == 0) nst = 1;
                for (int st = 0; st < nst; ++st, ++q) {
                    const uint32_t h = q & 1u;
                    if (!mbar_wait(smem_u32(&full_bar[h]), (q >> 1) & 1u)) { failed = true; break; }
                    if (q >= 1 && !mbar_wait(smem_u32(&free_bar), (q - 1) & 1u)) { failed = true; break; }
                    mbar_arrive(smem_u32(&stage_bar));
                    tc_fence_after();
                    const OzStage& S = stages[q % EXP_SLOTS];
                    if (!(S.flags & 4)) {
#pragma unroll
                        for (int g = 0; g < NORD; ++g) {
                            const uint32_t dt = tmem + (uint32_t)(g * OTN);
#pragma unroll
                            for (int i = 0; i <= g; ++i) {
                                const int j = g - i;
#pragma unroll
                                for (int kk = 0; kk < OTK / 16; ++kk) {
                                    const uint32_t koff = (h * (OTK / 16) + kk) * 32;
                                    const uint64_t ad = sdesc(sA + i * A_SLICE + koff, 16, 1024);
                                    const uint64_t bd = sdesc(sB + j * B_SLICE + koff, 16, 1024);
                                    mma_bf16(dt, ad, bd, id, (i == 0 && kk == 0) ? 0u : 1u);
                                }
                            }
                        }
                    }
                    mma_commit(smem_u32(&mma_bar[h]));
                }
            }
            mma_commit(smem_u32(&drain_bar));
            if (!mbar_wait(smem_u32(&drain_bar), 0)) failed = true;
        }
    } else {
        // ---------------- epilogue ----------------
        const int quarter = warp & 3, chalf = warp >> 2;
        const int row = quarter * 32 + lane;
        uint32_t q = 0;
        for (int it = blockIdx.x; it < total && !failed; it += gridDim.x) {
            const Tile T = tiles[it / nvec];
            const int v = it % nvec;
            int nst = tile_nst(T, segs);
            if (nst == 0) nst = 1;
            float ach[EPI_COLS];
            float* acl = acl_s + tid;  // acl[c * NEPI * 32]
#pragma unroll
            for (int c = 0; c < EPI_COLS; ++c) {
                ach[c] = 0.f;
                acl[c * NEPI * 32] = 0.f;
            }
            for (int st = 0; st < nst; ++st, ++q) {
                int ok = 1;
                if (lane == 0)
                    ok = (mbar_wait(smem_u32(&stage_bar), q & 1u) &&
                          mbar_wait(smem_u32(&mma_bar[q & 1u]), (q >> 1) & 1u))
                             ? 1
                             : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) { failed = true; break; }
                __syncwarp();
                tc_fence_after();
                const OzStage& S = stages[q % EXP_SLOTS];
                if (S.flags & 4) {
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&free_bar));
                    continue;
                }
                const int er = S.ea[row];
                const float ah = S.ah, al = S.al;
                const bool unit = (ah == 1.f || ah == -1.f) && al == 0.f;  // alpha = +-1: a sign only
                const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(chalf * EPI_COLS);
#pragma unroll
                for (int cc = 0; cc < EPI_COLS / 4; ++cc) {
                    uint32_t a[NORD][4];
#pragma unroll
                    for (int g = 0; g < NORD; ++g) tmem_ld4(tbase + (uint32_t)(g * OTN + cc * 4), a[g]);
                    tmem_wait_ld();
                    if (cc == EPI_COLS / 4 - 1) {  // every order of this stage is in registers: release the accumulators
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(smem_u32(&free_bar));
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int c = cc * 4 + j;
                        // sum of the orders, order g weighted 2^-8g, as a double-float
                        float sh = __uint_as_float(a[0][j]), sl = 0.f, e;
#pragma unroll
                        for (int g = 1; g < NORD; ++g) {
                            two_sum(sh, __uint_as_float(a[g][j]) * pow2f(-8 * g), sh, e);
                            sl += e;
                        }
                        // unit of order 0: 2^(E_r - 8) 2^(E_c - 8)
                        const float sc = pow2f(er + S.eb[chalf * EPI_COLS + c] - 16);
                        sh *= sc;
                        sl *= sc;
                        float p, pe;
                        if (unit) {
                            p = sh * ah;
                            pe = sl * ah;
                        } else {  // times alpha (double-float product)
                            p = sh * ah;
                            pe = fmaf(sh, ah, -p);
                            pe = fmaf(sh, al, pe);
                            pe = fmaf(sl, ah, pe);
                        }
                        float nh;
                        two_sum(ach[c], p, nh, e);
                        ach[c] = nh;
                        acl[c * NEPI * 32] += e + pe;
                    }
                }
            }
            if (failed) break;
            // the tile's FP64 result
            const int r = T.m0 + row;
            const int c0 = T.n0 + chalf * EPI_COLS;
            if (r < T.m && c0 < T.n) {
                const int ncol = min(EPI_COLS, T.n - c0);
                double* C = bt.p[T.c_buf] + T.c_off + (int64_t)v * bt.vstride[T.c_buf] + (int64_t)r * T.ldc + c0;
                if (T.mode == TILE_ATOMIC) {
#pragma unroll
                    for (int c = 0; c < EPI_COLS; ++c)
                        if (c < ncol) atomicAdd(C + c, (double)ach[c] + (double)acl[c * NEPI * 32]);
                } else {
#pragma unroll
                    for (int c = 0; c < EPI_COLS; ++c)
                        if (c < ncol) C[c] = (double)ach[c] + (double)acl[c * NEPI * 32];
                }
            }
        }
    }
    if (failed) atomicExch(err, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace

int oz_tile_rows() { return OTM; }
int oz_tile_cols() { return OTN; }
int oz_stage_depth() { return OTK; }

int* oz_error_word() {
    static int* d = nullptr;
    if (!d) {
        DMRG_CHECK_CUDA(cudaMalloc(&d, sizeof(int)));
        DMRG_CHECK_CUDA(cudaMemset(d, 0, sizeof(int)));
    }
    return d;
}

bool oz_take_error(cudaStream_t st) {
    int* d = oz_error_word();
    int h = 0;
    DMRG_CHECK_CUDA(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st));
    DMRG_CHECK_CUDA(cudaStreamSynchronize(st));
    if (h) DMRG_CHECK_CUDA(cudaMemsetAsync(d, 0, sizeof(int), st));
    return h != 0;
}

void launch_seg_gemm_oz(const WorkList& w, const BufTable& bt, int nvec, int* d_err, cudaStream_t st) {
    if (w.tiles.empty()) return;
    DMRG_REQUIRE(w.tile_m == OTM && w.tile_n == OTN, DMRG_EINVAL, "work list not lowered for the FP64 tensor-core engine");
    DMRG_REQUIRE(bt.pmask == 0, DMRG_EINVAL, "the FP64 tensor-core engine reads FP64 buffers only");
    const int64_t total = (int64_t)w.tiles.size() * nvec;
    DMRG_REQUIRE(total < (1LL << 31), DMRG_EINVAL, "work list too large for one launch");
    static bool attr = false;
    if (!attr) {
        DMRG_CHECK_CUDA(cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
        attr = true;
    }
    int dev = 0, nsm = 0;
    DMRG_CHECK_CUDA(cudaGetDevice(&dev));
    DMRG_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = (int)std::min<int64_t>(total, std::max(nsm, 1));
    oz_gemm_kernel<<<grid, OZ_THREADS, OZ_SMEM, st>>>(w.d_tiles, (int)w.tiles.size(), nvec, w.d_segs, bt, d_err);
    ++launch_counter();
    DMRG_CHECK_CUDA(cudaGetLastError());
}

}  // namespace dmrg

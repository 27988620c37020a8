// Tensor-core (tcgen05, sm_103a) segmented grouped GEMM on bf16 operand pieces.
#pragma once

#include <cuda.h>  // CUtensorMap (the encoder is fetched from the driver at run time)
#include <cuda_bf16.h>

#include <map>
#include <tuple>
#include <unordered_map>

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
    int64_t pstride[kMaxBufs];  // three pieces: piece 2 at lo + pstride
    int64_t vstride[kMaxBufs];
    void* out[kMaxBufs];       // double* / float* / bf16 hi pieces (by mode)
    void* out_lo[kMaxBufs];    // bf16 lo pieces for TC_STORE_SPLIT
    int64_t out_pstride[kMaxBufs];
    int64_t out_vstride[kMaxBufs];
    int* counter;              // dynamic tile counter (zeroed before each launch)
    int* err;                  // device error word (0 = ok)
};

// Launch over the tiles of `w` (Seg::alpha must be +1 or -1: a sign applied
// through the MMA negate bit; Tile::alpha scales the epilogue).
void launch_seg_gemm_tc(const WorkList& w, const TcBufs& b, int nvec, int nsplit, cudaStream_t st);

int tc_num_sms();
// one-time kernel attributes (dynamic shared memory) of the nsplit kernels
void tc_prepare(int nsplit);

// ---------------------------------------------------------------------------
// TMA-staged variant: every operand is addressed through a tensor map.
// ---------------------------------------------------------------------------

// A segment whose operands are read through tensor maps.  Each map is 4-D over
// one bf16 piece: x = column, y = row, z = operator row of a stored family
// (0 otherwise), w = vector index (for per-vector buffers).  The maps of a key
// come in piece order (hi, lo, lo2) at 3 * key + piece.
struct TSeg {
    int32_t a_map, b_map;  // map keys
    int32_t a_z, b_z;      // z coordinates
    int32_t k;             // K extent of the segment
    uint8_t a_tr, b_tr;    // a_tr: A held as K x M (MN-major); b_tr: B held as N x K (K-major)
    uint8_t a_pv, b_pv;    // 1: the operand's w coordinate is the vector index
    uint8_t a_br, b_br;    // rows of the maps' boxes (min(64, rows rounded up to 16))
    uint8_t pad[2];
    float sign;            // +1 or -1 (MMA negate bit)
};

struct TmaWorkList {
    std::vector<Tile> tiles;
    std::vector<TSeg> segs;
    Tile* d_tiles = nullptr;
    TSeg* d_segs = nullptr;
    size_t cap_tiles = 0, cap_segs = 0;
    // output block (m x n, ld ldc) at c_off of c_buf, 128 x tn tiles (tn = 64 or
    // 128), split into K-chunks of at most kchunk (atomic modes only)
    void add_block(int64_t c_off, int c_buf, int m, int n, int ldc, const std::vector<TSeg>& s, uint8_t mode,
                   int64_t kchunk, float alpha, int tn = 128);
    void order_tiles();  // longest tiles first (stable)
    void upload(cudaStream_t st);
    void release();
};

// A matrix as a tensor-map key: element (z, y, x) of vector w of buffer `buf`
// lives at off + w*vstride + z*zstride + y*ld + x (elements), x < cols, y < rows.
// Its boxes are 64 columns x box_rows(rows) rows.
inline int box_rows(int64_t rows) { return rows >= 64 ? 64 : (int)((rows + 15) / 16 * 16); }
struct MapKey {
    int buf;
    int64_t off;
    int64_t cols, rows, ld, nz, zstride, nv, vstride;
    auto tie() const { return std::tie(buf, off, cols, rows, ld, nz, zstride, nv, vstride); }
    bool operator<(const MapKey& o) const { return tie() < o.tie(); }
};

struct MapKeyHash {
    size_t operator()(const MapKey& k) const {
        uint64_t h = 0x9e3779b97f4a7c15ull ^ (uint64_t)k.buf;
        const int64_t v[9] = {k.off, k.cols, k.rows, k.ld, k.nz, k.zstride, k.nv, k.vstride, 0};
        for (int i = 0; i < 8; ++i) {
            h ^= (uint64_t)v[i] + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
            h *= 0xff51afd7ed558ccdull;
        }
        return (size_t)(h ^ (h >> 33));
    }
};
struct MapKeyEq {
    bool operator()(const MapKey& a, const MapKey& b) const { return a.tie() == b.tie(); }
};

struct MapTable {
    std::vector<MapKey> keys;
    std::unordered_map<MapKey, int, MapKeyHash, MapKeyEq> index;
    CUtensorMap* d_maps = nullptr;
    size_t cap = 0;
    const void* enc_ptr[kMaxBufs][3] = {};  // piece pointers the device maps were encoded with
    int get(const MapKey& k);  // validates alignment; returns the key index
    bool stale(const TcBufs& tb) const;  // a piece pointer moved since the last encode
    // encode 3 maps per key (pieces hi, lo, lo + pstride) and copy them to the device
    void encode_upload(const TcBufs& tb, int nsplit, cudaStream_t st);
    void clear() {
        keys.clear();
        index.clear();
    }
    void release();
};

// Launch the TMA-staged kernel over the tiles of `w` (maps on the device).
void launch_seg_gemm_tma(const TmaWorkList& w, const MapTable& maps, const TcBufs& b, int nvec, int nsplit,
                         cudaStream_t st);

// FP64 (unpadded rows of length n, ld_src) -> bf16 pieces (rows padded to ld_dst);
// lo2 (optional) receives the third piece x - hi - lo
void dev_split_f64(const double* src, int64_t rows, int n, int64_t ld_src, __nv_bfloat16* hi,
                   __nv_bfloat16* lo, int64_t ld_dst, cudaStream_t st, __nv_bfloat16* lo2 = nullptr);
// FP64 -> bf16 pieces, same layout, n elements
void dev_split_f64_flat(const double* src, int64_t n, __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t st,
                        __nv_bfloat16* lo2 = nullptr);
// FP32 -> bf16 pieces, same layout, n elements
void dev_split_f32(const float* src, int64_t n, __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t st,
                   __nv_bfloat16* lo2 = nullptr);
// batched block copy FP64 -> pieces: for each job (src_off, dst_off, rows, cols, ld_src, ld_dst)
struct SplitJob {
    int64_t src_off, dst_off;
    int rows, cols, ld_src, ld_dst;
};
void dev_split_blocks(const double* src, const SplitJob* d_jobs, int njobs, __nv_bfloat16* hi, __nv_bfloat16* lo,
                      cudaStream_t st, __nv_bfloat16* lo2 = nullptr);

}  // namespace dmrg

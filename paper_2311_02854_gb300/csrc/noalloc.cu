// dmrg_grouped_gemm_noalloc: the FP64 segmented grouped GEMM with its work
// list held in a fixed, statically allocated device array instead of memory
// obtained from cudaMalloc.
//
// Some callers cannot allocate device memory at the point where they need a
// product: a process that has handed all device memory to its own pool (a
// caching allocator, a serving runtime that reserves HBM up front) would see
// the allocation fail or force the pool to give memory back, and cudaFree
// synchronises the whole device, which stalls every other stream of a caller
// that overlaps work.  This entry point lets such callers run the same kernel
// with no device allocation and no device-wide synchronisation.
//
// Scratch: the tiles and segments of the work list are copied into
// g_worklist_scratch (kScratchBytes).  Its device address is looked up once per
// device, with that device current, by the first call made on it (under lazy
// module loading the driver places the array in device memory at that moment);
// that first call should therefore come before any stream capture begins.  Every call
// rewrites the scratch, so two calls whose executions overlap (different
// streams, or different host threads without ordering) race on it; calls on
// one stream are ordered and safe.
#include <cstring>
#include <mutex>

#include "engine.h"

namespace dmrg {
namespace {

constexpr int64_t kScratchBytes = 4 << 20;  // 4 MiB: work-list tiles + segments
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_worklist_scratch[kScratchBytes];

std::mutex g_setup_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once per device).
unsigned char* scratch_for_current_device() {
    int dev = 0;
    DMRG_CHECK_CUDA(cudaGetDevice(&dev));
    DMRG_REQUIRE(dev >= 0 && dev < kMaxDevices, DMRG_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_worklist_scratch);
        if (e != cudaSuccess || !p)
            throw Error(DMRG_ECUDA, std::string("scratch symbol lookup failed: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = (unsigned char*)p;
    }
    return g_scratch_ptr[dev];
}

}  // namespace

int64_t noalloc_scratch_bytes() { return kScratchBytes; }

// Work list of the product (host side) -> static scratch -> FP64 segmented GEMM.
void grouped_gemm_f64_noalloc(const WorkList& host_wl, const double* a, const double* b, double* c, cudaStream_t st) {
    if (host_wl.tiles.empty()) return;
    const int64_t tile_bytes = (int64_t)(host_wl.tiles.size() * sizeof(Tile));
    const int64_t seg_off = round_up(tile_bytes, 256);
    const int64_t seg_bytes = (int64_t)(host_wl.segs.size() * sizeof(Seg));
    const int64_t need = seg_off + seg_bytes;
    if (need > kScratchBytes)
        throw Error(DMRG_EINVAL, "work list needs " + std::to_string(need) + " bytes of static scratch; the limit is " +
                                     std::to_string(kScratchBytes) + " (" + std::to_string(sizeof(Tile)) +
                                     " bytes per 64x64 output tile, " + std::to_string(sizeof(Seg)) +
                                     " per segment)");
    // The work list is copied from host memory that is freed when the call
    // returns; a captured copy would replay from that dead pointer, so a
    // stream under capture is refused before anything is enqueued.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    DMRG_CHECK_CUDA(cudaStreamIsCapturing(st, &cap));
    DMRG_REQUIRE(cap == cudaStreamCaptureStatusNone, DMRG_EINVAL,
                 "dmrg_grouped_gemm_noalloc called on a stream that is being captured");
    unsigned char* base = scratch_for_current_device();
    DMRG_CHECK_CUDA(cudaMemcpyAsync(base, host_wl.tiles.data(), tile_bytes, cudaMemcpyHostToDevice, st));
    if (seg_bytes > 0)
        DMRG_CHECK_CUDA(cudaMemcpyAsync(base + seg_off, host_wl.segs.data(), seg_bytes, cudaMemcpyHostToDevice, st));
    BufTable bt{};
    bt.p[0] = const_cast<double*>(a);
    bt.p[1] = const_cast<double*>(b);
    bt.p[2] = c;
    launch_seg_gemm_f64_lists((const Tile*)base, (int64_t)host_wl.tiles.size(), (const Seg*)(base + seg_off), bt, st);
}

}  // namespace dmrg

// Host tier of the renormalised environment blocks (Sec. 2.3: the operators
// of the blocks that the current bond does not use are kept off the GPU and
// brought back before they are needed).
//
// A sweep holds every left block of the sites behind it and every right block
// ahead of it, but one bond update reads two of them (left[k-1], right[k+1]).
// With the host tier the others live in pinned host memory: a block is copied
// out once after it is built (blocks never change afterwards, so later
// evictions only free the device arrays) on a copy stream that runs beside
// the Davidson iteration, and the block of the next bond is prefetched on the
// same stream.  The compute stream waits for a prefetch only where the block
// is used.  Copies, not the GPU's access to host memory, move the data: every
// kernel keeps reading HBM.
#include <algorithm>
#include <chrono>

#include "bond.h"

namespace dmrg {
namespace {

int64_t bytes_d(const Block& b) { return b.has_d ? b.n * 8 : 0; }
int64_t bytes_h(const Block& b) { return b.has_h ? b.n * 2 : 0; }
int64_t bytes_l(const Plan& P, const Block& b) { return b.has_l ? (int64_t)P.lo_pieces() * b.n * 2 : 0; }
int64_t host_need(const Plan& P, const Block& b) { return bytes_d(b) + bytes_h(b) + bytes_l(P, b); }

cudaStream_t copy_stream(Plan& P) {
    if (!P.copy_stream) DMRG_CHECK_CUDA(cudaStreamCreateWithFlags(&P.copy_stream, cudaStreamNonBlocking));
    return P.copy_stream;
}

cudaEvent_t make_event() {
    cudaEvent_t e;
    DMRG_CHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return e;
}

// pinned buffer of at least n bytes: the smallest pooled one that fits, else a new one
char* host_take(Plan& P, int64_t n, int64_t& cap) {
    int best = -1;
    for (int i = 0; i < (int)P.host_pool.size(); ++i)
        if (P.host_pool[i].second >= n && (best < 0 || P.host_pool[i].second < P.host_pool[best].second)) best = i;
    if (best >= 0) {
        char* p = P.host_pool[best].first;
        cap = P.host_pool[best].second;
        P.host_pool.erase(P.host_pool.begin() + best);
        return p;
    }
    void* p = nullptr;
    if (cudaHostAlloc(&p, (size_t)n, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        throw Error(DMRG_ENOMEM, "pinned host allocation of " + std::to_string(n >> 20) + " MiB failed");
    }
    P.host_bytes += n;
    P.stats.host_bytes = P.host_bytes;
    cap = n;
    return (char*)p;
}

void free_dev(Plan& P, Block& b) {
    P.free(b.d, b.n);
    P.free_bf16(b.h, b.n);
    P.free_lo(b.l, b.n);
    b.dev = false;
    b.evicting = false;
}

}  // namespace

void tier_out(Plan& P, Block& b) {
    if (!b.dev || b.evicting) return;
    if (!b.ev_use) b.ev_use = make_event();
    // the compute stream's last use of the block precedes the copy and the free
    DMRG_CHECK_CUDA(cudaEventRecord(b.ev_use, P.stream));
    if (!b.host_valid) {
        b.has_d = b.d != nullptr;
        b.has_h = b.h != nullptr;
        b.has_l = b.l != nullptr;
        const int64_t need = host_need(P, b);
        if (need > 0) {
            b.host = host_take(P, need, b.host_cap);
            cudaStream_t cs = copy_stream(P);
            DMRG_CHECK_CUDA(cudaStreamWaitEvent(cs, b.ev_use, 0));
            char* h = b.host;
            if (b.has_d) DMRG_CHECK_CUDA(cudaMemcpyAsync(h, b.d, bytes_d(b), cudaMemcpyDeviceToHost, cs));
            h += bytes_d(b);
            if (b.has_h) DMRG_CHECK_CUDA(cudaMemcpyAsync(h, b.h, bytes_h(b), cudaMemcpyDeviceToHost, cs));
            h += bytes_h(b);
            if (b.has_l) DMRG_CHECK_CUDA(cudaMemcpyAsync(h, b.l, bytes_l(P, b), cudaMemcpyDeviceToHost, cs));
            if (!b.ev_out) b.ev_out = make_event();
            DMRG_CHECK_CUDA(cudaEventRecord(b.ev_out, cs));
            P.stats.tier_out_bytes += need;
        }
        b.host_valid = true;
    }
    b.evicting = true;
}

void tier_drain(Plan& P, bool wait) {
    const auto t0 = std::chrono::steady_clock::now();
    auto drain = [&](std::vector<std::unique_ptr<Block>>& v) {
        for (auto& b : v)
            if (b && b->evicting) {
                // the copy out (if any) and the compute stream's last use are done
                bool done = true;
                for (cudaEvent_t e : {b->ev_out, b->ev_use}) {
                    if (!e) continue;
                    if (wait) {
                        DMRG_CHECK_CUDA(cudaEventSynchronize(e));
                    } else {
                        const cudaError_t r = cudaEventQuery(e);
                        if (r == cudaErrorNotReady) {
                            done = false;
                            break;
                        }
                        DMRG_CHECK_CUDA(r);
                    }
                }
                if (done) free_dev(P, *b);
            }
    };
    drain(P.left);
    drain(P.right);
    P.stats.ms_tier_wait += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

void tier_in(Plan& P, Block& b) {
    if (b.evicting) {  // still on the device: cancel the eviction
        b.evicting = false;
        return;
    }
    if (b.dev) return;
    DMRG_REQUIRE(b.host_valid, DMRG_EINVAL, "environment block has neither a device nor a host copy");
    if (b.has_d) b.d = P.alloc(b.n);
    if (b.has_h) b.h = P.alloc_bf16(b.n);
    if (b.has_l) b.l = P.alloc_lo(b.n);
    b.dev = true;
    cudaStream_t cs = copy_stream(P);
    // the eviction's copy wrote the host buffer (long done: its device arrays were freed after it)
    const char* h = b.host;
    if (b.has_d) DMRG_CHECK_CUDA(cudaMemcpyAsync(b.d, h, bytes_d(b), cudaMemcpyHostToDevice, cs));
    h += bytes_d(b);
    if (b.has_h) DMRG_CHECK_CUDA(cudaMemcpyAsync(b.h, h, bytes_h(b), cudaMemcpyHostToDevice, cs));
    h += bytes_h(b);
    if (b.has_l) DMRG_CHECK_CUDA(cudaMemcpyAsync(b.l, h, bytes_l(P, b), cudaMemcpyHostToDevice, cs));
    if (!b.ev_in) b.ev_in = make_event();
    DMRG_CHECK_CUDA(cudaEventRecord(b.ev_in, cs));
    b.fetching = true;
    P.stats.tier_in_bytes += host_need(P, b);
}

void tier_need(Plan& P, Block& b) {
    tier_in(P, b);
    if (b.fetching) {
        DMRG_CHECK_CUDA(cudaStreamWaitEvent(P.stream, b.ev_in, 0));
        b.fetching = false;
    }
}

void tier_release(Plan& P, Block& b) {
    // a copy may still read the device arrays or write the host buffer
    for (cudaEvent_t e : {b.ev_out, b.ev_use, b.ev_in})
        if (e) DMRG_CHECK_CUDA(cudaEventSynchronize(e));
    b.evicting = b.fetching = false;
    if (b.host) P.host_pool.push_back({b.host, b.host_cap});
    b.host = nullptr;
    b.host_cap = 0;
    b.host_valid = false;
    for (cudaEvent_t e : {b.ev_out, b.ev_use, b.ev_in})
        if (e) cudaEventDestroy(e);
    b.ev_out = b.ev_use = b.ev_in = nullptr;
}

void tier_destroy(Plan& P) {
    if (P.copy_stream) {
        cudaStreamSynchronize(P.copy_stream);
        cudaStreamDestroy(P.copy_stream);
        P.copy_stream = nullptr;
    }
    for (auto& x : P.host_pool) cudaFreeHost(x.first);
    P.host_pool.clear();
}

void tier_policy(Plan& P, int k, bool forward) {
    if (!P.opt.host_tier) return;
    const int K = P.K;
    const int next = forward ? k + 2 : k - 2;  // index of the block the next bond adds
    auto keep = [&](bool left_side, int m) {
        if (left_side) return m == k - 1 || (!forward && m == next);
        return m == k + 1 || (forward && m == next);
    };
    for (int m = 0; m <= K; ++m) {
        if (P.left[m] && !keep(true, m)) tier_out(P, *P.left[m]);
        if (P.right[m] && !keep(false, m)) tier_out(P, *P.right[m]);
    }
    if (forward && next <= K && P.right[next]) tier_in(P, *P.right[next]);
    if (!forward && next >= 0 && P.left[next]) tier_in(P, *P.left[next]);
}

}  // namespace dmrg

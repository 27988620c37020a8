// Runtime of libdmrg: MPS input/output, device memory, lowering of block
// products onto the segmented GEMM, environments (renormalisation, Eq.
// Renorm), the bond's intermediates and sigma (Eq. Sigma), diag(H_eff).
#include <algorithm>
#include <atomic>
#include <exception>
#include <thread>
#include <array>
#include <cmath>
#include <cstring>
#include <fstream>
#include <unordered_map>

#include "bond.h"
#include "plan.h"

namespace dmrg {

// ---------------------------------------------------------------------------
// MPS file (layout documented in include/dmrg.h / synthetic_inputs.write_mps)
// ---------------------------------------------------------------------------

bool MPSHost::read(const std::string& path, std::string& err) {
    std::ifstream f(path, std::ios::binary);
    if (!f) {
        err = "cannot open MPS file " + path;
        return false;
    }
    char magic[8];
    f.read(magic, 8);
    if (!f || std::memcmp(magic, "DMRGMPS1", 8) != 0) {
        err = "not an MPS file: " + path;
        return false;
    }
    int32_t hdr[4];
    f.read((char*)hdr, sizeof(hdr));
    K = hdr[0];
    N = hdr[1];
    twoS = hdr[2];
    center = hdr[3];
    if (K < 2 || K > 512) {
        err = "bad K in MPS file";
        return false;
    }
    bonds.assign(K + 1, {});
    for (int b = 0; b <= K; ++b) {
        int32_t n;
        f.read((char*)&n, 4);
        if (!f || n < 0 || n > 100000) {
            err = "bad bond table in MPS file";
            return false;
        }
        for (int i = 0; i < n; ++i) {
            int32_t s[3];
            f.read((char*)s, 12);
            bonds[b].push_back({s[0], s[1], s[2]});
        }
    }
    sites.assign(K + 1, {});
    for (int k = 1; k <= K; ++k) {
        int32_t nb;
        f.read((char*)&nb, 4);
        if (!f || nb < 0) {
            err = "bad site table in MPS file";
            return false;
        }
        for (int i = 0; i < nb; ++i) {
            int32_t key[3];
            f.read((char*)key, 12);
            if (!f || key[0] < 0 || key[0] >= (int)bonds[k - 1].size() || key[2] < 0 ||
                key[2] >= (int)bonds[k].size() || key[1] < 0 || key[1] > 3) {
                err = "bad block key in MPS file";
                return false;
            }
            int64_t cnt = (int64_t)bonds[k - 1][key[0]][2] * bonds[k][key[2]][2];
            std::vector<double> data(cnt);
            f.read((char*)data.data(), cnt * 8);
            if (!f) {
                err = "truncated MPS file";
                return false;
            }
            sites[k][{key[0], key[1], key[2]}] = std::move(data);
        }
    }
    return true;
}

bool MPSHost::write(const std::string& path) const {
    std::ofstream f(path, std::ios::binary);
    if (!f) return false;
    f.write("DMRGMPS1", 8);
    int32_t hdr[4] = {K, N, twoS, center};
    f.write((const char*)hdr, sizeof(hdr));
    for (int b = 0; b <= K; ++b) {
        int32_t n = (int32_t)bonds[b].size();
        f.write((const char*)&n, 4);
        for (auto& s : bonds[b]) {
            int32_t v[3] = {s[0], s[1], s[2]};
            f.write((const char*)v, 12);
        }
    }
    for (int k = 1; k <= K; ++k) {
        // canonical order: il, n, matching ir
        std::vector<std::pair<std::array<int, 3>, const std::vector<double>*>> blocks;
        std::map<std::pair<int, int>, int> ridx;
        for (int i = 0; i < (int)bonds[k].size(); ++i) ridx[{bonds[k][i][0], bonds[k][i][1]}] = i;
        for (int il = 0; il < (int)bonds[k - 1].size(); ++il)
            for (int n = 0; n < 4; ++n) {
                auto it = ridx.find({bonds[k - 1][il][0] + kSiteQN[n].n, bonds[k - 1][il][1] + kSiteQN[n].s});
                if (it == ridx.end()) continue;
                auto bt = sites[k].find({il, n, it->second});
                blocks.push_back({{il, n, it->second}, bt == sites[k].end() ? nullptr : &bt->second});
            }
        int32_t nb = (int32_t)blocks.size();
        f.write((const char*)&nb, 4);
        for (auto& b : blocks) {
            int32_t key[3] = {b.first[0], b.first[1], b.first[2]};
            f.write((const char*)key, 12);
            int64_t cnt = (int64_t)bonds[k - 1][key[0]][2] * bonds[k][key[2]][2];
            if (b.second) {
                f.write((const char*)b.second->data(), cnt * 8);
            } else {
                std::vector<double> z(cnt, 0.0);
                f.write((const char*)z.data(), cnt * 8);
            }
        }
    }
    return (bool)f;
}

// ---------------------------------------------------------------------------
// Device memory
// ---------------------------------------------------------------------------

double* Plan::alloc(int64_t n) {
    if (n <= 0) return nullptr;
    int64_t bytes = n * 8;
    DMRG_REQUIRE(budget <= 0 || dev_bytes + bytes <= budget, DMRG_ENOMEM,
                 "device budget exceeded (" + std::to_string((dev_bytes + bytes) >> 20) + " MiB)");
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(DMRG_ENOMEM, "cudaMalloc of " + std::to_string(bytes >> 20) + " MiB failed");
    }
    dev_bytes += bytes;
    stats.device_bytes = dev_bytes;
    stats.device_bytes_peak = std::max(stats.device_bytes_peak, dev_bytes);
    return (double*)p;
}

void Plan::free(double*& p, int64_t n) {
    if (p) {
        cudaFree(p);
        dev_bytes -= n * 8;
        stats.device_bytes = dev_bytes;
    }
    p = nullptr;
}

__nv_bfloat16* Plan::alloc_bf16(int64_t n) {
    if (n <= 0) return nullptr;
    int64_t bytes = round_up(n * 2, 256);
    DMRG_REQUIRE(budget <= 0 || dev_bytes + bytes <= budget, DMRG_ENOMEM,
                 "device budget exceeded (" + std::to_string((dev_bytes + bytes) >> 20) + " MiB)");
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(DMRG_ENOMEM, "cudaMalloc of " + std::to_string(bytes >> 20) + " MiB failed");
    }
    dev_bytes += bytes;
    stats.device_bytes = dev_bytes;
    stats.device_bytes_peak = std::max(stats.device_bytes_peak, dev_bytes);
    return (__nv_bfloat16*)p;
}

void Plan::free_bf16(__nv_bfloat16*& p, int64_t n) {
    if (p) {
        cudaFree(p);
        dev_bytes -= round_up(n * 2, 256);
        stats.device_bytes = dev_bytes;
    }
    p = nullptr;
}

void Plan::check_device_error() {
    if (oz && oz_take_error(stream))
        throw Error(DMRG_ETIMEOUT, "the FP64 tensor-core engine gave up waiting (device error word set)");
    if (!d_ctr) return;
    int err = 0;
    DMRG_CHECK_CUDA(cudaMemcpyAsync(&err, d_ctr + 1, sizeof(int), cudaMemcpyDeviceToHost, stream));
    DMRG_CHECK_CUDA(cudaStreamSynchronize(stream));
    if (err) {
        DMRG_CHECK_CUDA(cudaMemsetAsync(d_ctr + 1, 0, sizeof(int), stream));
        throw Error(DMRG_ETIMEOUT, "a tensor-core kernel gave up waiting (device error word set)");
    }
}

void Plan::drop_graphs() {
    for (auto& kv : sigma_graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    sigma_graphs.clear();
}

cudaEvent_t Plan::take_event() {
    if (!ev_pool.empty()) {
        cudaEvent_t e = ev_pool.back();
        ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    DMRG_CHECK_CUDA(cudaEventCreate(&e));
    return e;
}

void Plan::collect_sigma_times(bool wait) {
    size_t keep = 0;
    for (size_t i = 0; i < sig_pending.size(); ++i) {
        SigmaEvents& x = sig_pending[i];
        if (wait) DMRG_CHECK_CUDA(cudaEventSynchronize(x.b));
        else if (cudaEventQuery(x.b) != cudaSuccess) {
            sig_pending[keep++] = x;
            continue;
        }
        float ms = 0.f;
        DMRG_CHECK_CUDA(cudaEventElapsedTime(&ms, x.a, x.b));
        stats.ms_sigma_dev += ms;
        stats.sigma_flops_dev += x.flops;
        stats.sigma_stages_dev += x.stages;
        ++stats.sigma_timed;
        ev_pool.push_back(x.a);
        ev_pool.push_back(x.b);
    }
    sig_pending.resize(keep);
    cudaGetLastError();  // a not-ready query leaves no error behind
}

Plan::~Plan() {
    for (auto& x : sig_pending) {
        cudaEventDestroy(x.a);
        cudaEventDestroy(x.b);
    }
    for (auto e : ev_pool) cudaEventDestroy(e);
    drop_graphs();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (d_sig_io) free(d_sig_io, n_sig_io);
    for (auto* side : {&left, &right})
        for (auto& b : *side)
            if (b) {
                try {
                    tier_release(*this, *b);
                } catch (...) {
                }
                if (b->d) free(b->d, b->n);
                free_bf16(b->h, b->n);
                free_lo(b->l, b->n);
            }
    tier_destroy(*this);
    free_bf16(s_hi, n_spc);
    free_lo(s_lo, n_spc);
    free_bf16(ps_hi, n_ppc);
    free_lo(ps_lo, n_ppc);
    free_bf16(id_hi, (int64_t)id_n * id_n);
    free_lo(id_lo, (int64_t)id_n * id_n);
    free_bf16(w_hi, n_wpc);
    free_lo(w_lo, n_wpc);
    if (d_psi_jobs) cudaFree(d_psi_jobs);
    mlp.release();
    if (d_mlp_feat) cudaFree(d_mlp_feat);
    if (d_ctr) cudaFree(d_ctr);
    sigma_tc.release();
    free(interm.d, interm.n);
    free_bf16(interm.h, interm.n);
    free_lo(interm.l, interm.n);
    free(d_scratch, n_scratch);
    free(d_ident, (int64_t)ident_n * ident_n);
    free(d_wcoef, n_wcoef);
    free(d_io, n_io);
    free(d_dav, n_dav);
    free(d_guess, n_guess);
    sigma_pl.release();
    sigma_units_pl.release();
    hdiag_pl.release();
}

// ---------------------------------------------------------------------------
// Lowering of three-factor products
// ---------------------------------------------------------------------------

void ProductList::clear() {
    release();
    outs.clear();
    cs.clear();
    chunks.clear();
    tchunks.clear();
    flops = 0.0;
    scratch_elems = 0;
}

void ProductList::release() {
    for (auto& c : chunks) {
        c.first.release();
        c.second.release();
    }
    for (auto& c : tchunks) {
        c.first.release();
        c.second.release();
    }
    maps.release();
}

static Seg make_seg(const View& A, const View& B, int k, double alpha) {
    Seg s{};
    s.a_off = A.off;
    s.b_off = B.off;
    s.k = k;
    s.lda = A.ld;
    s.ldb = B.ld;
    s.a_buf = (uint8_t)A.buf;
    s.b_buf = (uint8_t)B.buf;
    s.a_tr = A.tr;
    s.b_tr = B.tr;
    s.alpha = alpha;
    return s;
}

void ProductList::lower(int8_t sbuf_, int8_t ibuf, int ild, int64_t cap, int64_t kchunk) {
    const int8_t sbuf = sbuf_;
    this->sbuf = sbuf_;
    release();
    chunks.clear();
    flops = 0.0;
    scratch_elems = 0;
    size_t i = 0;
    auto ident_view = [&](void) {
        View v;
        v.buf = ibuf;
        v.off = 0;
        v.ld = ild;
        return v;
    };
    while (i < cs.size()) {
        WorkList p1, p2;
        p1.tile_m = p2.tile_m = tile_m;
        p1.tile_n = p2.tile_n = tile_n;
        std::vector<std::vector<Seg>> segs(outs.size());
        std::vector<char> seen(outs.size(), 0);
        std::vector<int> order;
        int64_t used = 0;
        for (; i < cs.size(); ++i) {
            const Contrib& c = cs[i];
            int nreal = (!c.P.ident) + (!c.Q.ident) + (!c.R.ident);
            int64_t need = 0;
            bool pq_first = true;
            if (nreal == 3) {
                double cost_pq = 2.0 * c.m * c.k1 * c.k2 + 2.0 * c.m * c.k2 * c.n;
                double cost_qr = 2.0 * c.k1 * c.k2 * c.n + 2.0 * c.m * c.k1 * c.n;
                pq_first = cost_pq <= cost_qr;
                need = pq_first ? (int64_t)c.m * c.k2 : (int64_t)c.k1 * c.n;
                need = round_up(need, 4);
                if (used + need > cap && used > 0) break;
                flops += std::min(cost_pq, cost_qr);
            }
            if (!seen[c.out]) {
                seen[c.out] = 1;
                order.push_back(c.out);
            }
            std::vector<Seg>& sv = segs[c.out];
            if (nreal == 3) {
                View T;
                T.buf = sbuf;
                T.off = used;
                if (pq_first) {
                    T.ld = c.k2;
                    std::vector<Seg> one{make_seg(c.P, c.Q, c.k1, 1.0)};
                    p1.add_block(used, sbuf, c.m, c.k2, c.k2, one, TILE_STORE);
                    sv.push_back(make_seg(T, c.R, c.k2, c.alpha));
                } else {
                    T.ld = c.n;
                    std::vector<Seg> one{make_seg(c.Q, c.R, c.k2, 1.0)};
                    p1.add_block(used, sbuf, c.k1, c.n, c.n, one, TILE_STORE);
                    sv.push_back(make_seg(c.P, T, c.k1, c.alpha));
                }
                used += need;
            } else if (nreal == 2) {
                if (c.P.ident) sv.push_back(make_seg(c.Q, c.R, c.k2, c.alpha));
                else if (c.R.ident) sv.push_back(make_seg(c.P, c.Q, c.k1, c.alpha));
                else sv.push_back(make_seg(c.P, c.R, c.k1, c.alpha));
                flops += 2.0 * c.m * c.n * (c.P.ident ? c.k2 : c.k1);
            } else {
                const View& F = !c.P.ident ? c.P : (!c.Q.ident ? c.Q : c.R);
                if (nreal == 1) sv.push_back(make_seg(F, ident_view(), c.n, c.alpha));
                else sv.push_back(make_seg(ident_view(), ident_view(), c.n, c.alpha));
                flops += 2.0 * c.m * c.n;
            }
        }
        for (int o : order) {
            const OutBlock& ob = outs[o];
            p2.add_block(ob.off, ob.buf, ob.m, ob.n, ob.ldc, segs[o], TILE_ATOMIC, kchunk);
        }
        scratch_elems = std::max(scratch_elems, used);
        chunks.emplace_back(std::move(p1), std::move(p2));
    }
}

void ProductList::lower_tc(int8_t sbuf_, int8_t ibuf, int ild, int64_t cap, int64_t kchunk, uint8_t out_mode) {
    const int8_t sbuf = sbuf_;
    this->sbuf = sbuf_;
    release();
    chunks.clear();
    flops = 0.0;
    scratch_elems = 0;
    tc = true;
    View I;
    I.buf = ibuf;
    I.off = 0;
    I.ld = ild;
    // scratch elements of a contribution's phase-1 product
    auto need_of = [&](const Contrib& c) -> int64_t {
        const int nreal = (!c.P.ident) + (!c.Q.ident) + (!c.R.ident);
        const bool unit = (c.alpha == 1.0 || c.alpha == -1.0);
        if (nreal == 3) {
            const double cost_pq = 2.0 * c.m * c.k1 * c.k2 + 2.0 * c.m * c.k2 * c.n;
            const double cost_qr = 2.0 * c.k1 * c.k2 * c.n + 2.0 * c.m * c.k1 * c.n;
            return cost_pq <= cost_qr ? (int64_t)c.m * round_up(c.k2, 8) : (int64_t)c.k1 * round_up(c.n, 8);
        }
        return unit ? 0 : (int64_t)c.m * round_up(c.n, 8);
    };
    // chunk boundaries: each chunk's phase-1 products fit the scratch
    std::vector<size_t> starts{0};
    {
        int64_t used = 0;
        for (size_t i = 0; i < cs.size(); ++i) {
            const int64_t need = need_of(cs[i]);
            if (used + need > cap && used > 0) {
                starts.push_back(i);
                used = 0;
            }
            used += need;
        }
    }
    starts.push_back(cs.size());
    const size_t nch = cs.empty() ? 0 : starts.size() - 1;
    // scratch offset of every contribution's phase-1 product inside its chunk
    std::vector<int64_t> soff(cs.size() + 1, 0);
    std::vector<int64_t> cused(nch, 0);
    for (size_t ch = 0; ch < nch; ++ch) {
        int64_t used = 0;
        for (size_t i = starts[ch]; i < starts[ch + 1]; ++i) {
            soff[i] = used;
            used += need_of(cs[i]);
        }
        cused[ch] = used;
    }
    // the chunks' items in units of at most kUnit on host threads: each unit's
    // phase-1 blocks and, per output, its phase-2 segments; concatenated per
    // chunk in item order (the result of lowering the items one by one)
    constexpr size_t kUnit = 8192;
    struct Unit {
        size_t ch, a, b;
        WorkList p1;
        std::vector<std::pair<int, Seg>> osegs;
        double fl = 0.0;
    };
    std::vector<Unit> units;
    std::vector<size_t> unit_beg(nch + 1, 0);
    for (size_t ch = 0; ch < nch; ++ch) {
        unit_beg[ch] = units.size();
        for (size_t a = starts[ch]; a < starts[ch + 1]; a += kUnit) {
            Unit u;
            u.ch = ch;
            u.a = a;
            u.b = std::min(starts[ch + 1], a + kUnit);
            units.push_back(std::move(u));
        }
    }
    unit_beg[nch] = units.size();
    parallel_for(units.size(), [&](size_t ui) {
        Unit& u = units[ui];
        WorkList& p1 = u.p1;
        double fl = 0.0;
        for (size_t i = u.a; i < u.b; ++i) {
            const Contrib& c = cs[i];
            const int nreal = (!c.P.ident) + (!c.Q.ident) + (!c.R.ident);
            const bool unit = (c.alpha == 1.0 || c.alpha == -1.0);
            const int64_t used = soff[i];
            bool pq_first = true;
            double cost = 0.0;
            int tc_ = 0;  // columns of the phase-1 product
            if (nreal == 3) {
                const double cost_pq = 2.0 * c.m * c.k1 * c.k2 + 2.0 * c.m * c.k2 * c.n;
                const double cost_qr = 2.0 * c.k1 * c.k2 * c.n + 2.0 * c.m * c.k1 * c.n;
                pq_first = cost_pq <= cost_qr;
                cost = std::min(cost_pq, cost_qr);
                tc_ = pq_first ? c.k2 : c.n;
            } else if (!unit) {
                tc_ = c.n;
            }
            View T;
            T.buf = sbuf;
            T.off = used;
            T.ld = (int)round_up(std::max(tc_, 1), 8);
            if (nreal == 3) {
                fl += cost;
                if (pq_first) {
                    p1.add_block(used, sbuf, c.m, c.k2, T.ld, {make_seg(c.P, c.Q, c.k1, 1.0)}, TC_STORE_SPLIT, 0, 128,
                                 (float)c.alpha);
                    u.osegs.push_back({c.out, make_seg(T, c.R, c.k2, 1.0)});
                } else {
                    p1.add_block(used, sbuf, c.k1, c.n, T.ld, {make_seg(c.Q, c.R, c.k2, 1.0)}, TC_STORE_SPLIT, 0, 128,
                                 (float)c.alpha);
                    u.osegs.push_back({c.out, make_seg(c.P, T, c.k1, 1.0)});
                }
                continue;
            }
            // the two (or one) real factors X (m x k) and Y (k x n)
            View X, Y;
            int k;
            if (nreal == 2) {
                if (c.P.ident) {
                    X = c.Q;
                    Y = c.R;
                    k = c.k2;
                } else if (c.R.ident) {
                    X = c.P;
                    Y = c.Q;
                    k = c.k1;
                } else {
                    X = c.P;
                    Y = c.R;
                    k = c.k1;
                }
                fl += 2.0 * c.m * c.n * k;
            } else {
                X = !c.P.ident ? c.P : (!c.Q.ident ? c.Q : c.R);
                Y = I;
                k = c.n;
                fl += 2.0 * c.m * c.n;
            }
            if (unit) {
                u.osegs.push_back({c.out, make_seg(X, Y, k, c.alpha)});
            } else {
                p1.add_block(used, sbuf, c.m, c.n, T.ld, {make_seg(X, Y, k, 1.0)}, TC_STORE_SPLIT, 0, 128,
                             (float)c.alpha);
                u.osegs.push_back({c.out, make_seg(T, I, c.n, 1.0)});
            }
        }
        u.fl = fl;
    });
    std::vector<std::pair<WorkList, WorkList>> built(nch);
    std::vector<double> cfl(nch, 0.0);
    parallel_for(nch, [&](size_t ch) {
        WorkList& p1 = built[ch].first;
        WorkList& p2 = built[ch].second;
        std::vector<std::vector<Seg>> segs(outs.size());
        std::vector<char> seen(outs.size(), 0);
        std::vector<int> order;
        for (size_t ui = unit_beg[ch]; ui < unit_beg[ch + 1]; ++ui) {
            Unit& u = units[ui];
            const int so = (int)p1.segs.size();
            for (Tile t : u.p1.tiles) {
                t.seg_beg += so;
                t.seg_end += so;
                p1.tiles.push_back(t);
            }
            p1.segs.insert(p1.segs.end(), u.p1.segs.begin(), u.p1.segs.end());
            p1.flops += u.p1.flops;
            for (const auto& os : u.osegs) {
                if (!seen[os.first]) {
                    seen[os.first] = 1;
                    order.push_back(os.first);
                }
                segs[os.first].push_back(os.second);
            }
            cfl[ch] += u.fl;
            u.p1 = WorkList();
            std::vector<std::pair<int, Seg>>().swap(u.osegs);
        }
        for (int o : order) {
            const OutBlock& ob = outs[o];
            p2.add_block(ob.off, ob.buf, ob.m, ob.n, ob.ldc, segs[o], out_mode, kchunk, 128, 1.0f);
        }
    });
    for (size_t ch = 0; ch < nch; ++ch) {
        flops += cfl[ch];
        scratch_elems = std::max(scratch_elems, cused[ch]);
        chunks.emplace_back(std::move(built[ch]));
    }
}

// ---------------------------------------------------------------------------
// TMA-staged lowering
// ---------------------------------------------------------------------------

namespace {

// Tensor-map key of view V read as a rows x cols matrix (before any transpose).
MapKey view_key(const View& V, int64_t rows, int64_t cols, const int64_t* vstride, int nv) {
    DMRG_REQUIRE(V.buf >= 0 && V.buf < kMaxBufs && !V.ident, DMRG_EINVAL, "tensor map of an implicit operand");
    MapKey k{};
    k.buf = V.buf;
    k.off = V.off - (int64_t)V.z * V.zstride;
    k.cols = cols;
    k.rows = rows;
    k.ld = V.ld;
    k.nz = V.nz;
    k.zstride = V.nz > 1 ? V.zstride : round_up(rows * V.ld, 8);
    const bool pv = vstride && vstride[V.buf] > 0;
    k.nv = pv ? nv : 1;
    k.vstride = pv ? vstride[V.buf] : k.nz * k.zstride;
    return k;
}

// out (m x n) += sign * op(A) (m x k) * op(B) (k x n) through tensor maps
TSeg make_tseg(MapTable& mt, const View& A, const View& B, int m, int n, int k, double sign, const int64_t* vstride,
               int nv) {
    TSeg s{};
    const MapKey ka = view_key(A, A.tr ? k : m, A.tr ? m : k, vstride, nv);
    const MapKey kb = view_key(B, B.tr ? n : k, B.tr ? k : n, vstride, nv);
    s.a_map = mt.get(ka);
    s.b_map = mt.get(kb);
    s.a_br = (uint8_t)box_rows(ka.rows);
    s.b_br = (uint8_t)box_rows(kb.rows);
    s.a_z = A.z;
    s.b_z = B.z;
    s.k = k;
    s.a_tr = A.tr;
    s.b_tr = B.tr;
    s.a_pv = (vstride && vstride[A.buf] > 0) ? 1 : 0;
    s.b_pv = (vstride && vstride[B.buf] > 0) ? 1 : 0;
    s.sign = sign < 0.0 ? -1.0f : 1.0f;
    return s;
}

}  // namespace

void ProductList::lower_tma(int8_t sbuf_, int8_t ibuf, int ild, int64_t cap, int64_t kchunk, uint8_t out_mode,
                            const int64_t* vstride_in, int nv, int tile_n) {
    const int8_t sbuf = sbuf_;
    this->sbuf = sbuf_;
    release();
    tchunks.clear();
    maps.clear();
    flops = 0.0;
    scratch_elems = 0;
    tc = true;
    View I;
    I.buf = ibuf;
    I.off = 0;
    I.ld = ild;
    // per-vector strides; the scratch holds one copy per vector, its stride (the
    // largest chunk's need) is set once the chunks are known
    int64_t vstride[kMaxBufs];
    for (int b = 0; b < kMaxBufs; ++b) vstride[b] = vstride_in ? vstride_in[b] : 0;
    vstride[sbuf] = round_up(std::max<int64_t>(cap, 8), 8);
    struct Item {
        int kind = 0;  // 3: three factors; 2: scaled two-factor product; 1: direct segment
        bool pq_first = true;
        int tr = 0, tcl = 0;  // phase-1 product rows / columns
        int grp = -1, z = 0;
        View X, Y;            // direct / scaled two-factor operands
        int k = 0;
        double fl = 0.0;  // algorithmic FLOPs of a kind 1 / 2 item
    };
    // pass 1 (sequential): the chunks of the list (each fits the scratch), the
    // items of each, their phase-1 shapes and scratch groups
    struct ChunkPlan {
        size_t i = 0, j = 0;
        std::vector<Item> items;
        std::vector<std::array<int64_t, 4>> groups;  // rows, cols, count, base
        int64_t used = 0;
    };
    std::vector<ChunkPlan> plans;
    size_t i = 0;
    while (i < cs.size()) {
        ChunkPlan cp;
        cp.i = i;
        std::unordered_map<int64_t, int> gidx;  // (rows << 32 | cols) -> scratch group
        size_t j = i;
        for (; j < cs.size(); ++j) {
            const Contrib& c = cs[j];
            if (chunk_per_term && j > i && c.term != cs[i].term) break;
            const int nreal = (!c.P.ident) + (!c.Q.ident) + (!c.R.ident);
            const bool unit = (c.alpha == 1.0 || c.alpha == -1.0);
            Item it;
            if (nreal == 3) {
                const double cost_pq = 2.0 * c.m * c.k1 * c.k2 + 2.0 * c.m * c.k2 * c.n;
                const double cost_qr = 2.0 * c.k1 * c.k2 * c.n + 2.0 * c.m * c.k1 * c.n;
                it.kind = 3;
                it.pq_first = cost_pq <= cost_qr;
                it.tr = it.pq_first ? c.m : c.k1;
                it.tcl = it.pq_first ? c.k2 : c.n;
            } else {
                if (nreal == 2) {
                    if (c.P.ident) {
                        it.X = c.Q;
                        it.Y = c.R;
                        it.k = c.k2;
                    } else if (c.R.ident) {
                        it.X = c.P;
                        it.Y = c.Q;
                        it.k = c.k1;
                    } else {
                        it.X = c.P;
                        it.Y = c.R;
                        it.k = c.k1;
                    }
                    it.fl = 2.0 * c.m * c.n * it.k;
                } else {
                    it.X = !c.P.ident ? c.P : (!c.Q.ident ? c.Q : c.R);
                    it.Y = I;
                    it.k = c.n;
                    it.fl = 2.0 * c.m * c.n;
                }
                it.kind = unit ? 1 : 2;
                if (!unit) {
                    it.tr = c.m;
                    it.tcl = c.n;
                }
            }
            int64_t need = 0;
            if (it.kind >= 2) need = (int64_t)it.tr * round_up(it.tcl, 8);
            if (cp.used + need > cap && cp.used > 0) break;
            if (it.kind >= 2) {
                const int64_t key = ((int64_t)it.tr << 32) | (int64_t)it.tcl;
                auto g = gidx.find(key);
                if (g == gidx.end()) {
                    g = gidx.emplace(key, (int)cp.groups.size()).first;
                    cp.groups.push_back({(int64_t)it.tr, (int64_t)it.tcl, 0, 0});
                }
                it.grp = g->second;
                it.z = (int)cp.groups[it.grp][2]++;
            }
            cp.used += need;
            cp.items.push_back(it);
        }
        int64_t base = 0;
        for (auto& g : cp.groups) {
            g[3] = base;
            base += g[2] * g[0] * round_up(g[1], 8);
        }
        cp.j = j;
        plans.push_back(std::move(cp));
        i = j;
    }
    // pass 2: the work lists.  Each chunk's items are cut into units of at
    // most kUnit items that run on host threads, each with a tensor-map table
    // of its own: a unit's phase-1 tiles and, per output block, its phase-2
    // segments.  The units' tables are merged into `maps` in order, and each
    // chunk's lists are concatenated from its units in order, so that the
    // result is that of lowering the items one by one.
    constexpr size_t kUnit = 8192;
    const size_t nch = plans.size();
    struct Unit {
        size_t ch, a, b;  // items [a, b) of chunk ch
        MapTable lm;
        TmaWorkList p1;
        std::vector<std::pair<int, TSeg>> osegs;  // (output block, phase-2 segment), item order
        double fl = 0.0;
    };
    std::vector<Unit> units;
    std::vector<size_t> unit_beg(nch + 1, 0);
    for (size_t ch = 0; ch < nch; ++ch) {
        unit_beg[ch] = units.size();
        const size_t ni = plans[ch].items.size();
        for (size_t a = 0; a < std::max<size_t>(ni, 1); a += kUnit) {
            Unit u;
            u.ch = ch;
            u.a = a;
            u.b = std::min(ni, a + kUnit);
            units.push_back(std::move(u));
        }
    }
    unit_beg[nch] = units.size();
    parallel_for(units.size(), [&](size_t ui) {
        Unit& u = units[ui];
        const ChunkPlan& cp = plans[u.ch];
        MapTable& lm = u.lm;
        TmaWorkList& p1 = u.p1;
        double fl = 0.0;
        for (size_t q = u.a; q < u.b; ++q) {
            const Contrib& c = cs[cp.i + q];
            const Item& it = cp.items[q];
            View T;
            if (it.kind >= 2) {
                const auto& g = cp.groups[it.grp];
                T.buf = sbuf;
                T.ld = (int)round_up(g[1], 8);
                T.zstride = g[0] * T.ld;
                T.nz = (int)g[2];
                T.z = it.z;
                T.off = g[3] + (int64_t)it.z * T.zstride;
            }
            if (it.kind == 3) {
                if (it.pq_first) {
                    fl += 2.0 * c.m * c.k1 * c.k2 + 2.0 * c.m * c.k2 * c.n;
                    p1.add_block(T.off, sbuf, c.m, c.k2, T.ld, {make_tseg(lm, c.P, c.Q, c.m, c.k2, c.k1, 1.0, vstride, nv)},
                                 TC_STORE_SPLIT, 0, (float)c.alpha, tile_n);
                    u.osegs.push_back({c.out, make_tseg(lm, T, c.R, c.m, c.n, c.k2, 1.0, vstride, nv)});
                } else {
                    fl += 2.0 * c.k1 * c.k2 * c.n + 2.0 * c.m * c.k1 * c.n;
                    p1.add_block(T.off, sbuf, c.k1, c.n, T.ld, {make_tseg(lm, c.Q, c.R, c.k1, c.n, c.k2, 1.0, vstride, nv)},
                                 TC_STORE_SPLIT, 0, (float)c.alpha, tile_n);
                    u.osegs.push_back({c.out, make_tseg(lm, c.P, T, c.m, c.n, c.k1, 1.0, vstride, nv)});
                }
            } else if (it.kind == 2) {
                fl += it.fl;
                p1.add_block(T.off, sbuf, c.m, c.n, T.ld, {make_tseg(lm, it.X, it.Y, c.m, c.n, it.k, 1.0, vstride, nv)},
                             TC_STORE_SPLIT, 0, (float)c.alpha, tile_n);
                u.osegs.push_back({c.out, make_tseg(lm, T, I, c.m, c.n, c.n, 1.0, vstride, nv)});
            } else {
                fl += it.fl;
                u.osegs.push_back({c.out, make_tseg(lm, it.X, it.Y, c.m, c.n, it.k, c.alpha, vstride, nv)});
            }
        }
        u.fl = fl;
    });
    // merge the units' map tables in order (sequential: first-seen order of the keys)
    std::vector<std::vector<int>> gi(units.size());
    for (size_t ui = 0; ui < units.size(); ++ui) {
        gi[ui].resize(units[ui].lm.keys.size());
        for (size_t x = 0; x < gi[ui].size(); ++x) gi[ui][x] = maps.get(units[ui].lm.keys[x]);
    }
    parallel_for(units.size(), [&](size_t ui) {
        Unit& u = units[ui];
        for (TSeg& sg : u.p1.segs) {
            sg.a_map = gi[ui][sg.a_map];
            sg.b_map = gi[ui][sg.b_map];
        }
        for (auto& os : u.osegs) {
            os.second.a_map = gi[ui][os.second.a_map];
            os.second.b_map = gi[ui][os.second.b_map];
        }
        u.lm.clear();
    });
    // per chunk (in parallel): phase 1 = the units' tiles in order; phase 2 =
    // one block per output with its segments in item order, outputs in the
    // order of their first item
    std::vector<TmaWorkList> w1(nch), w2(nch);
    std::vector<double> cfl(nch, 0.0);
    parallel_for(nch, [&](size_t ch) {
        TmaWorkList& p1 = w1[ch];
        TmaWorkList& p2 = w2[ch];
        size_t nt = 0, ns = 0;
        for (size_t ui = unit_beg[ch]; ui < unit_beg[ch + 1]; ++ui) {
            nt += units[ui].p1.tiles.size();
            ns += units[ui].p1.segs.size();
        }
        p1.tiles.reserve(nt);
        p1.segs.reserve(ns);
        std::vector<std::vector<TSeg>> segs(outs.size());
        std::vector<char> seen(outs.size(), 0);
        std::vector<int> order;
        for (size_t ui = unit_beg[ch]; ui < unit_beg[ch + 1]; ++ui) {
            Unit& u = units[ui];
            const int so = (int)p1.segs.size();
            for (Tile t : u.p1.tiles) {
                t.seg_beg += so;
                t.seg_end += so;
                p1.tiles.push_back(t);
            }
            p1.segs.insert(p1.segs.end(), u.p1.segs.begin(), u.p1.segs.end());
            for (const auto& os : u.osegs) {
                if (!seen[os.first]) {
                    seen[os.first] = 1;
                    order.push_back(os.first);
                }
                segs[os.first].push_back(os.second);
            }
            cfl[ch] += u.fl;
            u.p1 = TmaWorkList();
            std::vector<std::pair<int, TSeg>>().swap(u.osegs);
        }
        for (int o : order) {
            const OutBlock& ob = outs[o];
            p2.add_block(ob.off, ob.buf, ob.m, ob.n, ob.ldc, segs[o], out_mode, kchunk, 1.0f, tile_n);
        }
        p1.order_tiles();
        p2.order_tiles();
    });
    for (size_t ch = 0; ch < nch; ++ch) {
        flops += cfl[ch];
        scratch_elems = std::max(scratch_elems, plans[ch].used);
        tchunks.emplace_back(std::move(w1[ch]), std::move(w2[ch]));
    }
    // the scratch's per-vector stride is now known
    scratch_elems = round_up(std::max<int64_t>(scratch_elems, 8), 8);
    for (MapKey& k : maps.keys)
        if (k.buf == sbuf) k.vstride = scratch_elems;
    maps.index.clear();
}

void ProductList::run_tma(const TcBufs& tb, int nvec, int nsplit, cudaStream_t st) {
    for (auto& c : tchunks) {
        DMRG_REQUIRE(c.first.tiles.empty() || (sbuf >= 0 && tb.out[sbuf]), DMRG_EINVAL,
                     "tensor-core product list run without its scratch buffer");
        launch_seg_gemm_tma(c.first, maps, tb, nvec, nsplit, st);
        launch_seg_gemm_tma(c.second, maps, tb, nvec, nsplit, st);
    }
}

void ProductList::run_tc(const TcBufs& tb, int nvec, int nsplit, cudaStream_t st) {
    for (auto& c : chunks) {
        DMRG_REQUIRE(c.first.tiles.empty() || (sbuf >= 0 && tb.hi[sbuf] && tb.out[sbuf]), DMRG_EINVAL,
                     "tensor-core product list run without its scratch buffer");
        launch_seg_gemm_tc(c.first, tb, nvec, nsplit, st);
        launch_seg_gemm_tc(c.second, tb, nvec, nsplit, st);
    }
}

void ProductList::upload(cudaStream_t st) {
    for (auto& c : chunks) {
        c.first.upload(st);
        c.second.upload(st);
    }
}

void ProductList::run(const BufTable& bt, int nvec, cudaStream_t st) {
    for (auto& c : chunks) {
        DMRG_REQUIRE(c.first.tiles.empty() || (sbuf >= 0 && bt.p[sbuf]), DMRG_EINVAL,
                     "product list run without its scratch buffer");
        launch_seg_gemm_f64(c.first, bt, nvec, st);
        launch_seg_gemm_f64(c.second, bt, nvec, st);
    }
}

}  // namespace dmrg

// Shared host/device definitions of libdmrg: quantum numbers, sector bases,
// status handling and small utilities.
#pragma once

#include <cstdint>
#include <cstdio>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dmrg.h"

namespace dmrg {

// (particle number, 2*Sz) of a sector or the change made by an operator.
struct QN {
    int n = 0, s = 0;
    QN() = default;
    QN(int n_, int s_) : n(n_), s(s_) {}
    QN operator+(const QN& o) const { return {n + o.n, s + o.s}; }
    QN operator-(const QN& o) const { return {n - o.n, s - o.s}; }
    QN operator-() const { return {-n, -s}; }
    bool operator==(const QN& o) const { return n == o.n && s == o.s; }
    bool operator!=(const QN& o) const { return !(*this == o); }
    bool operator<(const QN& o) const { return n < o.n || (n == o.n && s < o.s); }
};

// Local basis of one spatial orbital: 0 vac, 1 beta, 2 alpha, 3 alpha-beta.
static const QN kSiteQN[4] = {{0, 0}, {1, -1}, {1, 1}, {2, 0}};

inline int spin_of(int p) { return (p % 2 == 0) ? 1 : -1; }  // 2*sz of spin orbital p

// Symmetry sectors of a block: own quantum numbers and dimensions.
struct Basis {
    std::vector<QN> qn;
    std::vector<int> dim;
    std::map<QN, int> index;
    void add(QN q, int d) {
        index[q] = (int)qn.size();
        qn.push_back(q);
        dim.push_back(d);
    }
    int find(QN q) const {
        auto it = index.find(q);
        return it == index.end() ? -1 : it->second;
    }
    int size() const { return (int)qn.size(); }
    int64_t total() const {
        int64_t t = 0;
        for (int d : dim) t += d;
        return t;
    }
    int dmax() const {
        int m = 0;
        for (int d : dim) m = d > m ? d : m;
        return m;
    }
};

struct Error : std::runtime_error {
    dmrg_status code;
    Error(dmrg_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define DMRG_CHECK_CUDA(call)                                                              \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            throw ::dmrg::Error(DMRG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define DMRG_REQUIRE(cond, code, msg)                       \
    do {                                                    \
        if (!(cond)) throw ::dmrg::Error((code), (msg));    \
    } while (0)

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace dmrg

// probe_color: torus colouring search of Sec. 3 (Eq. 15), host code.
//
// A colouring c(x) = sum_j sigma_j x_j mod n_c is distance-d valid on the
// torus iff no two distinct sites within wrap-around L1 distance d share a
// colour.  Two sites whose coordinates differ by the torus displacement D
// (D_j in [0, L_j)) differ in integer coordinates by e_j in {D_j, D_j - L_j}
// (both realised when D_j != 0), so validity means: sum_j sigma_j e_j is
// nonzero mod n_c for every such e.  Since e and -e give the same condition,
// one of each pair is kept.
//
// Search: n_c = 2, 3, ...; sigma walked in lexicographic order (sigma_1 most
// significant) depth first, carrying the partial sums sum_{i<=j} sigma_i e_i
// of every difference vector; a vector is tested at the depth of its last
// nonzero component, and a failing prefix is skipped with its subtree.  The
// first sigma reached is the lexicographically first valid one.
#include <stdint.h>
#include <string.h>

#include <vector>

#include "../../include/wd.h"

namespace {

struct Diffs {
    int nD;
    std::vector<std::vector<int>> byDepth;   // flattened e vectors (nD ints) whose last nonzero is at depth j
};

Diffs collect(const int *L, int nD, int d) {
    Diffs out;
    out.nD = nD;
    out.byDepth.assign(nD, std::vector<int>());
    std::vector<int> D(nD, 0);
    while (true) {
        // advance odometer (first coordinate fastest)
        int j = 0;
        while (j < nD) {
            if (++D[j] < L[j]) break;
            D[j] = 0;
            ++j;
        }
        if (j == nD) break;
        int dist = 0, last = -1;
        for (int i = 0; i < nD; ++i) {
            int a = D[i], b = L[i] - D[i];
            dist += a < b ? a : b;
            if (D[i]) last = i;
        }
        if (dist > d) continue;
        std::vector<int> nz;
        for (int i = 0; i < nD; ++i) if (D[i]) nz.push_back(i);
        for (unsigned w = 0; w < (1u << nz.size()); ++w) {
            std::vector<int> e(D.begin(), D.end());
            for (size_t k = 0; k < nz.size(); ++k) if (w >> k & 1) e[nz[k]] -= L[nz[k]];
            // keep one of e, -e: the one whose first nonzero component is positive
            int first = 0;
            for (int i = 0; i < nD; ++i) if (e[i]) { first = e[i]; break; }
            if (first < 0) continue;
            out.byDepth[last].insert(out.byDepth[last].end(), e.begin(), e.end());
        }
    }
    return out;
}

struct Walker {
    const Diffs &df;
    int nc;
    std::vector<int> sigma;
    std::vector<std::vector<long>> partial;   // partial[j][k]: sum_{i<=j} sigma_i e_i for all vectors of depth >= j

    Walker(const Diffs &d, int n) : df(d), nc(n), sigma(d.nD, 0) {}

    // all vectors listed once, with their depth
    bool run() {
        std::vector<const int *> vec;
        std::vector<int> depth;
        for (int j = 0; j < df.nD; ++j)
            for (size_t k = 0; k < df.byDepth[j].size(); k += df.nD) {
                vec.push_back(&df.byDepth[j][k]);
                depth.push_back(j);
            }
        std::vector<long> acc(vec.size(), 0);
        return step(0, vec, depth, acc);
    }

    bool step(int j, const std::vector<const int *> &vec, const std::vector<int> &depth, std::vector<long> &acc) {
        if (j == df.nD) return true;
        std::vector<long> next(acc.size());
        for (int s = 0; s < nc; ++s) {
            sigma[j] = s;
            bool ok = true;
            for (size_t k = 0; k < vec.size(); ++k) {
                if (depth[k] < j) continue;
                long v = acc[k] + (long)s * vec[k][j];
                next[k] = v;
                if (depth[k] == j && ((v % nc) + nc) % nc == 0) { ok = false; break; }
            }
            if (ok && step(j + 1, vec, depth, next)) return true;
        }
        return false;
    }
};

}  // namespace

extern "C" int probe_color(const int *dims, int nD, int d, int *n_colors, int *sigma, int32_t *colors) {
    if (!dims || !n_colors || !sigma || nD < 1 || nD > 4 || d < 0) return WD_EINVAL;
    long V = 1;
    for (int j = 0; j < nD; ++j) {
        if (dims[j] < 1) return WD_EINVAL;
        V *= dims[j];
    }
    Diffs df = collect(dims, nD, d);
    for (int nc = 2; nc <= 4096; ++nc) {
        Walker w(df, nc);
        if (!w.run()) continue;
        *n_colors = nc;
        for (int j = 0; j < nD; ++j) sigma[j] = w.sigma[j];
        if (colors) {
            std::vector<int> x(nD, 0);
            for (long i = 0; i < V; ++i) {
                long r = i, c = 0;
                for (int j = 0; j < nD; ++j) { x[j] = (int)(r % dims[j]); r /= dims[j]; c += (long)sigma[j] * x[j]; }
                colors[i] = (int32_t)(c % nc);
            }
        }
        return WD_OK;
    }
    return WD_ENOTSUP;
}

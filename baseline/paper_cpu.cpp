// The paper's own CPU algorithms for S^3TTVc on the CCSS forest (Sec. III-IV),
// kept as comparators for the GPU library: FP64, OpenMP over the host cores.
//
//   * Algorithm 3 (the paper's naive baseline): for every special leaf (e, v)
//     start from E_N(b_v) and walk from the leaf's owner up to its root,
//     convolving with Ebar_N(b_u) of every forest node on the way (full length-N
//     truncated products, no memoisation); atomically add the scaled degree-(N-1)
//     coefficient to s_v.  |e| - 1 products per leaf, |e|^2 - |e| per edge.
//   * Algorithm 4 (memoised): one depth-first traversal per tree; the truncated
//     product of Ebar_N over the path to the current node is kept per level, so
//     every forest edge costs one product and every special leaf one dot with
//     E_N(b_u).  Products are restricted to the degrees some special leaf below
//     still needs (the trimming the paper allows after Algorithm 4).
//
// Readings (the same as the rest of the project): the scale of a leaf is
// w(e) (N-1)! / |beta(e)| with w(e) = |e| and |beta(e)| = |e|! S(N, |e|) (the
// weight of Algorithm 3 with the edge size; Algorithm 4's printed weight is read
// the same way), and a child's product is the parent's truncated at degree N-1
// times Ebar_N of the child's vertex.  Nodes inside an edge are in increasing id
// order (the index order of Sec. II-B).
//
// Test and measurement infrastructure: it shares no code with the CUDA library
// or with the oracle.
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

namespace {

struct Forest {
    int32_t N = 0;
    int64_t n = 0;
    // nodes numbered level by level; the children of a node are contiguous
    std::vector<int32_t> vertex, level;
    std::vector<int64_t> parent, child_begin, child_end;
    std::vector<int64_t> leaf_begin, leaf_end;   // special leaves owned by the node
    std::vector<int32_t> top;                    // highest degree the node's product is needed at
    std::vector<int32_t> leaf_vertex;            // the dropped vertex of each special leaf
    std::vector<double> leaf_scale;              // w(e) (N-1)! / |beta(e)|
    std::vector<int64_t> roots;
    std::vector<int32_t> single_vertex;          // size-1 edges: s_v += b_v^(N-1)
    std::vector<double> single_scale;
    int64_t products3 = 0, products4 = 0;        // truncated products of Algorithms 3 and 4
};

// |e| (N-1)! / (|e|! S(N, |e|)) through R(n,k) = k! S(n,k) / n!, which satisfies
// R(n,k) = (k/n)(R(n-1,k) + R(n-1,k-1)), R(0,0) = 1: the scale is k / (N R(N,k)).
std::vector<double> leaf_scales(int N) {
    std::vector<double> R(N + 2, 0.0), Rn(N + 2, 0.0);
    R[0] = 1.0;
    for (int nn = 1; nn <= N; ++nn) {
        std::fill(Rn.begin(), Rn.end(), 0.0);
        for (int k = 1; k <= nn; ++k) Rn[k] = (double)k / nn * (R[k] + R[k - 1]);
        R.swap(Rn);
    }
    std::vector<double> sc(N + 1, 0.0);
    for (int k = 1; k <= N; ++k) sc[k] = (double)k / ((double)N * R[k]);
    return sc;
}

// Trimmed CCSS forest: every special leaf (e, v), |e| >= 2, owns the root-to-node
// path spelled by e minus v in increasing order; the forest holds exactly the
// nodes on such paths.  Built level by level by sorting (parent, vertex) keys.
Forest *build(int64_t n, int64_t m, const int64_t *ptr, const int32_t *mem, int32_t N) {
    Forest *f = new Forest();
    f->N = N;
    f->n = n;
    const std::vector<double> sc = leaf_scales(N);
    std::vector<int32_t> sorted(mem, mem + ptr[m]);
    for (int64_t e = 0; e < m; ++e) std::sort(sorted.begin() + ptr[e], sorted.begin() + ptr[e + 1]);
    struct Path {
        int64_t e;
        int32_t drop, len;
    };
    std::vector<Path> paths;
    for (int64_t e = 0; e < m; ++e) {
        const int32_t s = (int32_t)(ptr[e + 1] - ptr[e]);
        if (s == 1) {
            f->single_vertex.push_back(sorted[ptr[e]]);
            f->single_scale.push_back(sc[1]);
            continue;
        }
        for (int32_t i = 0; i < s; ++i) paths.push_back({e, i, s - 1});
    }
    auto elem = [&](const Path &p, int l) {  // l-th element (0-based) of e minus its dropped member
        return sorted[ptr[p.e] + (l < p.drop ? l : l + 1)];
    };
    std::vector<int64_t> at(paths.size(), -1);   // the path's node at the current level
    std::vector<int64_t> active(paths.size());
    std::iota(active.begin(), active.end(), 0);
    std::vector<std::vector<int64_t>> owned_by_level;   // per level: (node, path) pairs in node order
    std::vector<std::pair<uint64_t, int64_t>> keys;
    int64_t level_start = 0;
    for (int l = 1; !active.empty(); ++l) {
        keys.clear();
        for (int64_t pi : active) {
            const uint64_t par = l == 1 ? 0 : (uint64_t)(at[pi] - level_start + 1);
            keys.push_back({(par << 32) | (uint32_t)elem(paths[pi], l - 1), pi});
        }
        std::sort(keys.begin(), keys.end());
        const int64_t base = (int64_t)f->vertex.size();
        std::vector<int64_t> next;
        uint64_t last = ~0ull;
        for (auto &kv : keys) {
            if (kv.first != last) {
                last = kv.first;
                const int64_t par = l == 1 ? -1 : level_start + (int64_t)(kv.first >> 32) - 1;
                f->vertex.push_back((int32_t)(kv.first & 0xffffffffu));
                f->level.push_back(l);
                f->parent.push_back(par);
            }
            at[kv.second] = (int64_t)f->vertex.size() - 1;
            if (paths[kv.second].len > l) next.push_back(kv.second);
        }
        level_start = base;
        active.swap(next);
    }
    const int64_t nodes = (int64_t)f->vertex.size();
    // children: nodes of a level are sorted by parent, so each parent's children are contiguous
    f->child_begin.assign(nodes, 0);
    f->child_end.assign(nodes, 0);
    for (int64_t k = 0; k < nodes; ++k) {
        if (f->parent[k] < 0) {
            f->roots.push_back(k);
            continue;
        }
        int64_t p = f->parent[k];
        if (f->child_end[p] == 0) f->child_begin[p] = k;
        f->child_end[p] = k + 1;
    }
    // special leaves grouped by owner
    std::vector<int64_t> order(paths.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return at[a] < at[b]; });
    f->leaf_begin.assign(nodes, 0);
    f->leaf_end.assign(nodes, 0);
    for (size_t r = 0; r < order.size(); ++r) {
        const Path &p = paths[order[r]];
        const int64_t owner = at[order[r]];
        if (f->leaf_end[owner] == 0) f->leaf_begin[owner] = (int64_t)r;
        f->leaf_end[owner] = (int64_t)r + 1;
        f->leaf_vertex.push_back(sorted[ptr[p.e] + p.drop]);
        f->leaf_scale.push_back(sc[p.len + 1]);
        f->products3 += p.len;
    }
    // the highest degree each node's product is needed at: N-1 where the node owns leaves,
    // one less than its children's otherwise (a child at level l+1 needs its parent's
    // degrees up to its own top - 1); nodes come after their parents, so go backwards
    f->top.assign(nodes, -1);
    for (int64_t k = nodes - 1; k >= 0; --k) {
        if (f->leaf_end[k] > f->leaf_begin[k]) f->top[k] = N - 1;
        if (f->parent[k] >= 0) f->top[f->parent[k]] = std::max(f->top[f->parent[k]], f->top[k] - 1);
    }
    f->products4 = nodes - (int64_t)f->roots.size();
    return f;
}

// e^(b t) - 1 (bar = true) or e^(b t) on degrees 0..N-1
void egf(double b, int N, bool bar, double *out) {
    double t = 1.0;
    for (int k = 0; k < N; ++k) {
        out[k] = t;
        t = t * b / (double)(k + 1);
    }
    if (bar) out[0] = 0.0;
}

void atomic_add(double *p, double v) {
#pragma omp atomic
    *p += v;
}

}  // namespace

extern "C" {

void *pc_build(int64_t n, int64_t m, const int64_t *edge_ptr, const int32_t *members, int32_t N) {
    if (n < 1 || m < 0 || N < 1 || N > 128) return nullptr;
    return build(n, m, edge_ptr, members, N);
}

void pc_free(void *h) { delete static_cast<Forest *>(h); }

// info: nodes, roots, special leaves, levels, products of Algorithm 3, products of Algorithm 4
void pc_info(void *h, int64_t *info) {
    const Forest *f = static_cast<const Forest *>(h);
    info[0] = (int64_t)f->vertex.size();
    info[1] = (int64_t)f->roots.size();
    info[2] = (int64_t)f->leaf_vertex.size() + (int64_t)f->single_vertex.size();
    info[3] = f->level.empty() ? 0 : f->level.back();
    info[4] = f->products3;
    info[5] = f->products4;
}

// Special leaves (members) in the trees of roots [r0, r1).
int64_t pc_leaves_in_roots(void *h, int64_t r0, int64_t r1) {
    const Forest *f = static_cast<const Forest *>(h);
    int64_t cnt = 0;
    std::vector<int64_t> st;
    for (int64_t r = r0; r < r1; ++r) {
        st.assign(1, f->roots[r]);
        while (!st.empty()) {
            const int64_t v = st.back();
            st.pop_back();
            cnt += f->leaf_end[v] - f->leaf_begin[v];
            for (int64_t c = f->child_begin[v]; c < f->child_end[v]; ++c) st.push_back(c);
        }
    }
    return cnt;
}

// Algorithm 3 on the special leaves in the trees of roots [r0, r1) (all roots: r1 < 0),
// plus the size-1 edges when the whole forest is requested.  s (n doubles) is added to.
void pc_alg3(void *h, const double *b, double *s, int32_t nthreads, int64_t r0, int64_t r1) {
    const Forest *f = static_cast<const Forest *>(h);
    const int N = f->N;
    const bool all = r1 < 0;
    if (all) {
        r0 = 0;
        r1 = (int64_t)f->roots.size();
    }
    // the owners of the selected trees' leaves: collect node ranges per tree
    std::vector<int64_t> owners;
    {
        std::vector<int64_t> st;
        for (int64_t r = r0; r < r1; ++r) {
            st.assign(1, f->roots[r]);
            while (!st.empty()) {
                const int64_t v = st.back();
                st.pop_back();
                if (f->leaf_end[v] > f->leaf_begin[v]) owners.push_back(v);
                for (int64_t c = f->child_begin[v]; c < f->child_end[v]; ++c) st.push_back(c);
            }
        }
    }
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
        std::vector<double> coefs(N), ebar(N), tmp(N);
#pragma omp for schedule(dynamic, 64)
        for (int64_t oi = 0; oi < (int64_t)owners.size(); ++oi) {
            const int64_t owner = owners[oi];
            for (int64_t li = f->leaf_begin[owner]; li < f->leaf_end[owner]; ++li) {
                const int32_t v = f->leaf_vertex[li];
                egf(b[v], N, false, coefs.data());
                for (int64_t u = owner; u >= 0; u = f->parent[u]) {
                    egf(b[f->vertex[u]], N, true, ebar.data());
                    for (int j = 0; j < N; ++j) {
                        double acc = 0.0;
                        for (int k = 1; k <= j; ++k) acc += ebar[k] * coefs[j - k];
                        tmp[j] = acc;
                    }
                    coefs.swap(tmp);
                }
                atomic_add(&s[v], f->leaf_scale[li] * coefs[N - 1]);
            }
        }
        if (all) {
#pragma omp for
            for (int64_t i = 0; i < (int64_t)f->single_vertex.size(); ++i) {
                const int32_t v = f->single_vertex[i];
                atomic_add(&s[v], std::pow(b[v], (double)(N - 1)));
            }
        }
    }
}

// Algorithm 4 on the trees of roots [r0, r1) (all roots: r1 < 0, plus the size-1 edges).
void pc_alg4(void *h, const double *b, double *s, int32_t nthreads, int64_t r0, int64_t r1) {
    const Forest *f = static_cast<const Forest *>(h);
    const int N = f->N;
    const bool all = r1 < 0;
    if (all) {
        r0 = 0;
        r1 = (int64_t)f->roots.size();
    }
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
        // W[l]: the truncated product over the path to the current node at level l (degrees 0..N-1)
        std::vector<double> W((size_t)(N + 1) * N, 0.0), e(N);
        std::vector<std::pair<int64_t, int64_t>> st;   // (node, next child)
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = r0; r < r1; ++r) {
            const int64_t root = f->roots[r];
            double *P1 = &W[(size_t)1 * N];
            egf(b[f->vertex[root]], N, true, P1);
            st.assign(1, {root, f->child_begin[root]});
            bool enter = true;
            while (!st.empty()) {
                const int64_t v = st.back().first;
                const int l = f->level[v];
                const double *P = &W[(size_t)l * N];
                if (enter) {
                    // special leaves of v: dot of P with E_N(b_u) at total degree N-1
                    for (int64_t li = f->leaf_begin[v]; li < f->leaf_end[v]; ++li) {
                        const int32_t u = f->leaf_vertex[li];
                        egf(b[u], N, false, e.data());
                        double acc = 0.0;
                        for (int j = l; j <= N - 1; ++j) acc += P[j] * e[N - 1 - j];
                        atomic_add(&s[u], f->leaf_scale[li] * acc);
                    }
                    enter = false;
                }
                int64_t &next = st.back().second;
                if (next < f->child_end[v]) {
                    const int64_t c = next++;
                    // child's product: P times Ebar_N(b_c) on degrees l+1 .. top(c)
                    double *Q = &W[(size_t)(l + 1) * N];
                    const double bc = b[f->vertex[c]];
                    egf(bc, N, true, e.data());
                    const int topc = f->top[c];
                    for (int j = l + 1; j <= topc; ++j) {
                        double acc = 0.0;
                        for (int k = 1; k <= j - l; ++k) acc += e[k] * P[j - k];
                        Q[j] = acc;
                    }
                    st.push_back({c, f->child_begin[c]});
                    enter = true;
                } else {
                    st.pop_back();
                }
            }
        }
        if (all) {
#pragma omp for
            for (int64_t i = 0; i < (int64_t)f->single_vertex.size(); ++i) {
                const int32_t v = f->single_vertex[i];
                atomic_add(&s[v], std::pow(b[v], (double)(N - 1)));
            }
        }
    }
}

}  // extern "C"

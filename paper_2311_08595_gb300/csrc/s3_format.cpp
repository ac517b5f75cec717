// Host-side format builder: validation, index-ordered edges, size buckets,
// node-sorted incidence for the deterministic reduce, and the trimmed CCSS
// forest of Sec. III.  No CUDA calls here, so s3_format_inspect runs on any host.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <sstream>

#include "s3_internal.h"

namespace s3 {

// K(s,N) = w(e)/|beta(e)| * (N-1)! with w(e) = s and |beta(e)| = s! S(N,s)
// (Sec. II and its footnote).  Evaluated without cancellation through
// R(n,k) = k! S(n,k) / n!, which obeys R(n,k) = (k/n) (R(n-1,k) + R(n-1,k-1))
// with R(0,0) = 1 (all terms positive), so K = s / (N R(N,s)).
double scale_K(int s, int N) {
    std::vector<double> prev(N + 2, 0.0), cur(N + 2, 0.0);
    prev[0] = 1.0;  // R(0, 0)
    for (int n = 1; n <= N; ++n) {
        std::fill(cur.begin(), cur.end(), 0.0);
        for (int k = 1; k <= n; ++k) cur[k] = (double)k / (double)n * (prev[k] + prev[k - 1]);
        std::swap(prev, cur);
    }
    return (double)s / ((double)N * prev[s]);
}

// Rescaling target for one edge of size s at rank N.  The kernels multiply the
// edge's x values by an exact power of two g so that g * sum|x_u| is close to
// T(s,N).  T is chosen so that, for equal entries, the coefficient
// [t^(N-1)] (e^(a t) - 1)^s with a = T/s is about 1:
//   a^(N-1) s! S(N-1,s) / (N-1)! = 1,
// and a = 1 when s = N (then only the product of the other entries is
// needed).  This keeps every intermediate coefficient of the truncated series
// within a few decades of 1 in both FP32 and FP64.
float scale_target(int s, int N) {
    if (N <= 1) return 1.0f;
    if (s >= N) return (float)s;
    // log(s! S(N-1, s)) via log R(N-1, s) + log((N-1)!)
    std::vector<double> prev(N + 2, 0.0), cur(N + 2, 0.0);
    prev[0] = 1.0;
    for (int n = 1; n <= N - 1; ++n) {
        std::fill(cur.begin(), cur.end(), 0.0);
        for (int k = 1; k <= n; ++k) cur[k] = (double)k / (double)n * (prev[k] + prev[k - 1]);
        std::swap(prev, cur);
    }
    double R = prev[s];  // s! S(N-1,s) / (N-1)!
    if (!(R > 0.0)) return (float)s;
    double a = std::pow(1.0 / R, 1.0 / (double)(N - 1));
    return (float)(a * s);
}

s3_status build_host_format(int64_t n, int64_t m, const int64_t *edge_ptr, const int32_t *members,
                            const s3_options &opt, HostFormat &f) {
    if (n < 1) return fail(S3_EINVAL, "n must be >= 1");
    if (m < 0) return fail(S3_EINVAL, "m must be >= 0");
    if (!edge_ptr) return fail(S3_EINVAL, "edge_ptr is NULL");
    if (edge_ptr[0] != 0) return fail(S3_EINVAL, "edge_ptr[0] must be 0");
    if (n > INT32_MAX) return fail(S3_EINVAL, "n must fit int32 ids");
    int32_t max_edge = 0;
    for (int64_t e = 0; e < m; ++e) {
        int64_t sz = edge_ptr[e + 1] - edge_ptr[e];
        if (sz < 0) return fail(S3_EINVAL, "edge_ptr must be non-decreasing");
        if (sz == 0) {
            std::ostringstream os;
            os << "edge " << e << " is empty";
            return fail(S3_EINVAL, os.str());
        }
        if (sz > S3_MAX_RANK) return fail(S3_EINVAL, "edge larger than S3_MAX_RANK");
        max_edge = std::max<int32_t>(max_edge, (int32_t)sz);
    }
    const int64_t nnz = edge_ptr[m];
    if (nnz >= (int64_t)INT32_MAX) return fail(S3_EINVAL, "sum of edge sizes must be < 2^31");
    if (nnz > 0 && !members) return fail(S3_EINVAL, "members is NULL");
    int32_t N = opt.rank > 0 ? opt.rank : max_edge;
    if (N < 1) N = 1;
    if (N < max_edge) return fail(S3_EINVAL, "rank is smaller than the largest edge");
    if (N > S3_MAX_RANK) return fail(S3_EINVAL, "rank exceeds S3_MAX_RANK");
    for (int64_t j = 0; j < nnz; ++j)
        if (members[j] < 0 || members[j] >= n) {
            std::ostringstream os;
            os << "member " << j << " has id " << members[j] << " outside [0, n)";
            return fail(S3_EINVAL, os.str());
        }

    f = HostFormat();
    f.n = n;
    f.m = m;
    f.nnz = nnz;
    f.N = N;
    f.max_edge = max_edge;

    // node order inside edges: by decreasing degree (ties by id), or by id (index order)
    const bool by_degree = opt.order != S3_ORDER_INDEX;
    std::vector<int32_t> key_of;  // key_of[v]: position of v in the chosen order
    if (by_degree) {
        std::vector<int64_t> deg(n, 0);
        for (int64_t j = 0; j < nnz; ++j) deg[members[j]]++;
        std::vector<int32_t> order(n);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return deg[a] > deg[b]; });
        key_of.assign(n, 0);
        for (int64_t r = 0; r < n; ++r) key_of[order[r]] = (int32_t)r;
    }
    // sorted edges (as keys); reject repeats
    std::vector<int32_t> sorted(nnz);
    for (int64_t j = 0; j < nnz; ++j) sorted[j] = by_degree ? key_of[members[j]] : members[j];
    for (int64_t e = 0; e < m; ++e) {
        auto b = sorted.begin() + edge_ptr[e], t = sorted.begin() + edge_ptr[e + 1];
        std::sort(b, t);
        if (std::adjacent_find(b, t) != t) {
            std::ostringstream os;
            os << "edge " << e << " repeats a node";
            return fail(S3_EINVAL, os.str());
        }
    }
    // back from keys to node ids
    std::vector<int32_t> node_of_key;
    if (by_degree) {
        node_of_key.assign(n, 0);
        for (int64_t v = 0; v < n; ++v) node_of_key[key_of[v]] = (int32_t)v;
    }

    // size buckets
    std::vector<int64_t> count(N + 1, 0);
    for (int64_t e = 0; e < m; ++e) count[edge_ptr[e + 1] - edge_ptr[e]]++;
    std::vector<int64_t> bucket_of_size(N + 1, -1);
    int64_t off = 0;
    for (int s = 1; s <= N; ++s) {
        if (!count[s]) continue;
        HostBucket b;
        b.s = s;
        b.m = count[s];
        b.ld = (count[s] + 3) / 4 * 4;
        b.offset = off;
        off += (int64_t)s * b.ld;
        bucket_of_size[s] = (int64_t)f.buckets.size();
        f.buckets.push_back(b);
    }
    f.ids.assign(off, 0);
    f.slot.assign(off, 0);
    std::vector<int64_t> fillk(N + 1, 0);
    // edges of a bucket: lexicographic by key sequence (degree order) or input order
    std::vector<int64_t> edge_order(m);
    std::iota(edge_order.begin(), edge_order.end(), 0);
    if (by_degree) {
        std::stable_sort(edge_order.begin(), edge_order.end(), [&](int64_t a, int64_t b) {
            int64_t sa = edge_ptr[a + 1] - edge_ptr[a], sb = edge_ptr[b + 1] - edge_ptr[b];
            if (sa != sb) return sa < sb;
            const int32_t *pa = sorted.data() + edge_ptr[a], *pb = sorted.data() + edge_ptr[b];
            return std::lexicographical_compare(pa, pa + sa, pb, pb + sb);
        });
    }
    for (int64_t r = 0; r < m; ++r) {
        int64_t e = edge_order[r];
        int s = (int)(edge_ptr[e + 1] - edge_ptr[e]);
        const HostBucket &b = f.buckets[bucket_of_size[s]];
        int64_t k = fillk[s]++;
        for (int i = 0; i < s; ++i) {
            int32_t key = sorted[edge_ptr[e] + i];
            f.ids[b.offset + (int64_t)i * b.ld + k] = by_degree ? node_of_key[key] : key;
        }
    }

    // degrees (inc_ptr holds their prefix sums)
    f.inc_ptr.assign(n + 1, 0);
    for (int64_t j = 0; j < nnz; ++j) f.inc_ptr[members[j] + 1]++;
    for (int64_t v = 0; v < n; ++v) {
        f.max_degree = std::max(f.max_degree, f.inc_ptr[v + 1]);
        f.inc_ptr[v + 1] += f.inc_ptr[v];
    }

    // Layout of the per-(edge, node) buffer the reduce reads ("slots"):
    //  * nodes of degree <= kSmallDeg, sorted by decreasing degree (ties by id), form groups
    //    of 32; group g owns width_g * 32 slots from grp_off[g], and the k-th incidence of the
    //    group's lane-l node sits at grp_off[g] + 32 k + l (sliced ELL: a warp reads each k
    //    with one coalesced load; width_g is the group's largest degree, and the slots past
    //    a lane's own degree are padding that no kernel reads or writes);
    //  * then every medium node (degree <= kMedDeg) owns a contiguous segment
    //    (read by eight lanes up to kMed8Deg, by a warp above);
    //  * then every big node, cut into pieces of at most kPiece slots.
    // Inside a node, incidences are ordered by bucket, then edge, then member.
    std::vector<int64_t> base(n, 0);
    std::vector<int32_t> step(n, 1);
    {
        std::vector<int32_t> small;
        for (int64_t v = 0; v < n; ++v)
            if (f.inc_ptr[v + 1] - f.inc_ptr[v] <= kSmallDeg) small.push_back((int32_t)v);
        std::stable_sort(small.begin(), small.end(), [&](int32_t a, int32_t b) {
            return f.inc_ptr[a + 1] - f.inc_ptr[a] > f.inc_ptr[b + 1] - f.inc_ptr[b];
        });
        int64_t off = 0;
        for (size_t g0 = 0; g0 < small.size(); g0 += 32) {
            const int32_t w = (int32_t)(f.inc_ptr[small[g0] + 1] - f.inc_ptr[small[g0]]);
            f.grp_off.push_back(off);
            for (int l = 0; l < 32; ++l) {
                size_t i = g0 + l;
                f.grp_node.push_back(i < small.size() ? small[i] : -1);
                f.grp_deg.push_back(i < small.size() ? (uint8_t)(f.inc_ptr[small[i] + 1] - f.inc_ptr[small[i]]) : 0);
                if (i < small.size()) {
                    base[small[i]] = off + l;
                    step[small[i]] = 32;
                }
            }
            off += 32 * (int64_t)w;
        }
        for (int64_t v = 0; v < n; ++v) {
            int64_t d = f.inc_ptr[v + 1] - f.inc_ptr[v];
            if (d > kSmallDeg && d <= kMedDeg) {
                (d <= kMed8Deg ? f.med8_node : f.med_node).push_back((int32_t)v);
                (d <= kMed8Deg ? f.med8_off : f.med_off).push_back(off);
                (d <= kMed8Deg ? f.med8_len : f.med_len).push_back((int32_t)d);
                base[v] = off;
                off += d;
            }
        }
        for (int64_t v = 0; v < n; ++v) {
            int64_t d = f.inc_ptr[v + 1] - f.inc_ptr[v];
            if (d > kMedDeg) {
                f.big_node.push_back((int32_t)v);
                f.big_piece_ptr.push_back((int32_t)f.piece_start.size());
                base[v] = off;
                for (int64_t st = 0; st < d; st += kPiece) {
                    f.piece_start.push_back(off + st);
                    f.piece_big.push_back((int32_t)(f.big_node.size() - 1));
                    f.piece_len.push_back((int32_t)std::min<int64_t>(kPiece, d - st));
                }
                off += d;
            }
        }
        f.big_piece_ptr.push_back((int32_t)f.piece_start.size());
        f.buf_len = off;
    }
    if (f.buf_len >= (int64_t)INT32_MAX) return fail(S3_EINVAL, "incidence buffer exceeds 2^31 slots");
    {
        std::vector<int32_t> kth(n, 0);
        for (const HostBucket &b : f.buckets)
            for (int64_t k = 0; k < b.m; ++k)
                for (int i = 0; i < b.s; ++i) {
                    int64_t at = b.offset + (int64_t)i * b.ld + k;
                    int32_t v = f.ids[at];
                    f.slot[at] = (int32_t)(base[v] + (int64_t)step[v] * kth[v]++);
                }
    }

    // ------------------------------------------------------------- CCSS --
    if (!(opt.build_ccss || opt.layout == S3_LAYOUT_CCSS)) return S3_OK;
    f.has_ccss = true;
    HostCCSS &c = f.ccss;
    // One path per special leaf (e, v) with |e| >= 2: the sorted sequence e minus v.
    // paths are identified by (bucket, edge k, dropped member index i).
    struct PathRef { int32_t bucket; int32_t drop; int64_t k; };
    std::vector<PathRef> paths;
    paths.reserve(nnz);
    for (size_t bi = 0; bi < f.buckets.size(); ++bi) {
        const HostBucket &b = f.buckets[bi];
        if (b.s < 2) continue;
        for (int64_t k = 0; k < b.m; ++k)
            for (int i = 0; i < b.s; ++i) paths.push_back({(int32_t)bi, i, k});
    }
    auto path_elem = [&](const PathRef &p, int l) -> int32_t {  // l-th element (0-based) of the path
        const HostBucket &b = f.buckets[p.bucket];
        int i = l < p.drop ? l : l + 1;
        return f.ids[b.offset + (int64_t)i * b.ld + p.k];
    };
    auto path_len = [&](const PathRef &p) { return f.buckets[p.bucket].s - 1; };

    const int maxlev = std::max(0, max_edge - 1);
    std::vector<int32_t> node_of(paths.size(), -1);  // node id at the current level (level-local)
    std::vector<std::vector<int32_t>> lv_vertex(maxlev + 1), lv_parent(maxlev + 1);
    // per level: dedup (parent, vertex)
    std::vector<std::pair<uint64_t, int64_t>> keys;
    std::vector<int64_t> active(paths.size());
    std::iota(active.begin(), active.end(), 0);
    std::vector<int32_t> final_node(paths.size(), -1);        // node (level-local) at path end
    for (int l = 1; l <= maxlev; ++l) {
        keys.clear();
        std::vector<int64_t> next_active;
        for (int64_t pi : active) {
            const PathRef &p = paths[pi];
            if (path_len(p) < l) continue;
            uint32_t par = l == 1 ? 0u : (uint32_t)node_of[pi];
            uint32_t v = (uint32_t)path_elem(p, l - 1);
            keys.push_back({((uint64_t)par << 32) | v, pi});
        }
        if (keys.empty()) break;
        std::sort(keys.begin(), keys.end());
        int32_t id = -1;
        uint64_t last = ~0ull;
        for (auto &kv : keys) {
            if (kv.first != last) {
                ++id;
                last = kv.first;
                lv_vertex[l].push_back((int32_t)(kv.first & 0xffffffffu));
                lv_parent[l].push_back(l == 1 ? -1 : (int32_t)(kv.first >> 32));
            }
            node_of[kv.second] = id;
            if (path_len(paths[kv.second]) == l) final_node[kv.second] = id;
            else next_active.push_back(kv.second);
        }
        active.swap(next_active);
        c.levels = l;
    }
    // widths: own leaves, then children (bottom-up)
    std::vector<std::vector<int32_t>> lv_width(c.levels + 1);
    for (int l = 1; l <= c.levels; ++l) lv_width[l].assign(lv_vertex[l].size(), 0);
    for (size_t pi = 0; pi < paths.size(); ++pi) {
        int s = f.buckets[paths[pi].bucket].s;
        int l = s - 1;
        int32_t &w = lv_width[l][final_node[pi]];
        w = std::max<int32_t>(w, N - s + 1);
    }
    for (int l = c.levels; l >= 2; --l)
        for (size_t k = 0; k < lv_vertex[l].size(); ++k) {
            int32_t &pw = lv_width[l - 1][lv_parent[l][k]];
            pw = std::max(pw, lv_width[l][k]);
        }
    // reorder each level by width (descending, stable) and flatten
    std::vector<std::vector<int32_t>> new_index(c.levels + 1);
    c.level_begin.assign(1, 0);
    for (int l = 1; l <= c.levels; ++l) {
        size_t cnt = lv_vertex[l].size();
        std::vector<int32_t> order(cnt);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t a, int32_t b) { return lv_width[l][a] > lv_width[l][b]; });
        new_index[l].assign(cnt, 0);
        for (size_t r = 0; r < cnt; ++r) new_index[l][order[r]] = (int32_t)r;
        int64_t base = c.level_begin.back();
        for (size_t r = 0; r < cnt; ++r) {
            int32_t k = order[r];
            c.vertex.push_back(lv_vertex[l][k]);
            int32_t par = lv_parent[l][k];
            c.parent.push_back(l == 1 ? -1 : (int32_t)(c.level_begin[l - 2] + new_index[l - 1][par]));
            c.width.push_back(lv_width[l][k]);
        }
        c.level_begin.push_back(base + (int64_t)cnt);
        // width segments
        for (size_t r = 0; r < cnt;) {
            size_t q = r;
            int32_t w = lv_width[l][order[r]];
            while (q < cnt && lv_width[l][order[q]] == w) ++q;
            c.segs.push_back({l, w, base + (int64_t)r, base + (int64_t)q});
            r = q;
        }
    }
    c.value_off.resize(c.vertex.size());
    int64_t voff = 0;
    for (size_t k = 0; k < c.vertex.size(); ++k) {
        c.value_off[k] = voff;
        voff += c.width[k];
    }
    c.value_len = voff;
    c.products = (int64_t)c.vertex.size() - (c.levels >= 1 ? c.level_begin[1] : 0);
    // special leaves grouped by edge size
    std::vector<std::vector<int64_t>> by_s(N + 1);
    for (size_t pi = 0; pi < paths.size(); ++pi) by_s[f.buckets[paths[pi].bucket].s].push_back((int64_t)pi);
    for (int s = 2; s <= N; ++s) {
        if (by_s[s].empty()) continue;
        HostCCSS::LeafClass lc;
        lc.s = s;
        lc.begin = (int64_t)c.leaf_node.size();
        for (int64_t pi : by_s[s]) {
            const PathRef &p = paths[pi];
            const HostBucket &b = f.buckets[p.bucket];
            int l = s - 1;
            int64_t at = b.offset + (int64_t)p.drop * b.ld + p.k;
            c.leaf_node.push_back((int32_t)(c.level_begin[l - 1] + new_index[l][final_node[pi]]));
            c.leaf_vertex.push_back(f.ids[at]);
            c.leaf_slot.push_back(f.slot[at]);
        }
        lc.end = (int64_t)c.leaf_node.size();
        c.leaf_classes.push_back(lc);
    }
    return S3_OK;
}

void fill_info(const HostFormat &f, s3_format_info *info) {
    std::memset(info, 0, sizeof(*info));
    info->n = f.n;
    info->m = f.m;
    info->nnz = f.nnz;
    info->rank = f.N;
    info->max_edge = f.max_edge;
    info->max_degree = f.max_degree;
    for (const HostBucket &b : f.buckets) info->edges_per_size[b.s] = b.m;
    if (f.has_ccss) {
        const HostCCSS &c = f.ccss;
        info->ccss_levels = c.levels;
        for (int l = 1; l <= c.levels; ++l) info->ccss_nodes_per_level[l] = c.level_begin[l] - c.level_begin[l - 1];
        info->ccss_nodes = (int64_t)c.vertex.size();
        info->ccss_special_leaves = (int64_t)c.leaf_node.size();
        int64_t ones = f.buckets.size() && f.buckets[0].s == 1 ? f.buckets[0].m : 0;
        info->ccss_special_leaves += ones;  // size-1 edges hang below the (implicit) root
        info->ccss_products = c.products;
    }
}

}  // namespace s3

// Internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/s3ttvc.h"

namespace s3 {

// ------------------------------------------------------------------ errors --
void set_error(const std::string &msg);
s3_status fail(s3_status st, const std::string &msg);

// -------------------------------------------------------- host-side format --

// One size bucket: all edges with |e| = s, members stored "structure of arrays":
// member i of bucket edge k sits at ids[i * ld + k].
struct HostBucket {
    int32_t s = 0;
    int64_t m = 0;        // edges in the bucket
    int64_t ld = 0;       // leading dimension (m rounded up to a multiple of 4)
    int64_t offset = 0;   // offset of this bucket's arrays in the concatenated id/slot arrays
};

// The trimmed CCSS forest (Sec. III), level by level.  Level l (1-based) holds
// the distinct sorted prefixes of length l of the sequences e minus v.  Node k of
// level l stores its last node id, its parent (index into level l-1, -1 at
// level 1) and the width of the window of series coefficients it must keep
// (N - s_min + 1, s_min the smallest edge size of a special leaf below it).
// Nodes inside a level are sorted by width (descending) so that nodes of
// equal width are contiguous.
struct HostCCSS {
    int32_t levels = 0;
    std::vector<int64_t> level_begin;     // levels+1 offsets into the node arrays
    std::vector<int32_t> vertex, parent;  // per node
    std::vector<int32_t> width;           // per node
    std::vector<int64_t> value_off;       // per node: offset of its window in the value array
    int64_t value_len = 0;
    // width segments inside each level: (level, width, begin, end) node ranges
    struct Seg { int32_t level, width; int64_t begin, end; };
    std::vector<Seg> segs;
    // special leaves grouped by edge size s: leaf j of size class s is (node at level s-1,
    // dropped vertex, slot in node-sorted incidence order)
    struct LeafClass { int32_t s; int64_t begin, end; };
    std::vector<LeafClass> leaf_classes;
    std::vector<int32_t> leaf_node;       // index into the level s-1 node arrays (global index)
    std::vector<int32_t> leaf_vertex;
    std::vector<int32_t> leaf_slot;
    int64_t products = 0;                 // forest nodes at level >= 2
};

struct HostFormat {
    int64_t n = 0, m = 0, nnz = 0;
    int32_t N = 0, max_edge = 0;
    int64_t max_degree = 0;
    std::vector<HostBucket> buckets;      // non-empty buckets, increasing s
    std::vector<int32_t> ids;             // concatenated SoA member ids
    std::vector<int32_t> slot;            // same layout: position in node-sorted incidence order
    std::vector<int64_t> inc_ptr;         // n+1: prefix sums of the node degrees
    // deterministic reduce work lists over the slot buffer
    // small nodes (degree <= kSmallDeg): groups of 32 in sliced-ELL layout
    std::vector<int64_t> grp_off;         // first slot of each group
    std::vector<int32_t> grp_node;        // 32 per group, -1 = padding lane
    std::vector<uint8_t> grp_deg;         // 32 per group: the lane's degree (0 for padding)
    // medium nodes (kSmallDeg < degree <= kMedDeg), each a contiguous segment:
    // up to kMed8Deg eight lanes per node (med8_*), above one warp per node (med_*)
    std::vector<int32_t> med8_node, med8_len;
    std::vector<int64_t> med8_off;
    std::vector<int32_t> med_node, med_len;
    std::vector<int64_t> med_off;
    std::vector<int32_t> big_node;        // degree > kMedDeg (pieces of at most kPiece slots)
    int64_t buf_len = 0;                  // slots of the per-(edge, node) buffer (>= nnz)
    std::vector<int32_t> big_piece_ptr;   // pieces of big_node[k]: [big_piece_ptr[k], big_piece_ptr[k+1])
    std::vector<int64_t> piece_start;     // first slot of each piece
    std::vector<int32_t> piece_big;       // index into big_node of each piece's node
    std::vector<int32_t> piece_len;
    bool has_ccss = false;
    HostCCSS ccss;
};

constexpr int kSmallDeg = 32;
constexpr int kMed8Deg = 128;
constexpr int kMedDeg = 1024;
constexpr int kPiece = 2048;

s3_status build_host_format(int64_t n, int64_t m, const int64_t *edge_ptr, const int32_t *members,
                            const s3_options &opt, HostFormat &out);
void fill_info(const HostFormat &f, s3_format_info *info);

// Exact-in-spirit host tables: K(s,N) = s (N-1)! / (s! S(N,s)) in double and the
// per-edge rescaling target T(s,N) (see s3_format.cpp).
double scale_K(int s, int N);
float scale_target(int s, int N);

}  // namespace s3

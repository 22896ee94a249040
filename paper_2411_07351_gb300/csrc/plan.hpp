// Host plan builder: split tree, exact merge tables, fused-subtree programs,
// pass schedule and workspace layout for one (h, w, dtype, quadrants,
// boundary, split) request.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "fht_desc.h"

namespace fht {

enum class Split : int32_t { T = 0, S = 1 };

// Section 3: Split_T(n) = <2^(ceil(log2 n) - 1), rest>; Split_S(n) = <floor(n/2), ceil(n/2)>.
void split_sizes(int32_t n, Split rule, int32_t& n0, int32_t& n1);

// [a / d] for a >= 0, d > 0, ties to even; exact integer arithmetic.
int64_t round_half_even(int64_t a, int64_t d);

struct TreeNode {
  int32_t a = 0, m = 1;       // rows [a, a + m) of the view
  int32_t child[2] = {-1, -1};
  int32_t height = 0;         // 0 for a single row
  int32_t buf = -1;           // workspace buffer holding the node's Hough rows (-1: output)
};

struct Tree {
  int32_t n = 0;
  std::vector<TreeNode> nodes;  // children precede parents; the root is last
  int32_t root() const { return (int32_t)nodes.size() - 1; }
};

// Build G(n) of Theorem 1's proof: the binary tree of recursive splits.
Tree build_tree(int32_t n, Split rule);

// Merge table of a node of size m with children (m0, m1):
// t -> (t1, t2, s) with t1 = [t(m0-1)/(m-1)], t2 = [t(m1-1)/(m-1)], s = t - t2.
void merge_entry(int32_t m, int32_t m0, int32_t m1, int32_t t, int32_t& t1, int32_t& t2, int32_t& s);

// The whole table of one node, t = 0..m-1, computed without division: the
// quotient and remainder of t (m_i - 1) / (m - 1) are stepped as t grows.
struct MergeRow {
  int32_t t1, t2, s;
};
void merge_table(int32_t m, int32_t m0, int32_t m1, std::vector<MergeRow>& out);

struct PlanConfig {
  int32_t h = 0, w = 0;
  int32_t dtype = 0;       // fht_dtype
  uint32_t quads = 1;
  int32_t ext = 0;         // boundary
  Split split = Split::T;
  int32_t F = 64;          // fused rows
  int32_t TW = 0;          // fused column tile (0: the planner's default)
  int32_t threads = 0;     // fused CTA size (0: the planner's default)
  int32_t spine_chunk = 3; // spine nodes merged per spine-sum launch (the lower chunks first)
  int32_t generic_cols = 0; // column tile of generic subtrees (0: half of TW, at least 32)
  bool with_adjoint = false;  // also build the adjoint tables
  int32_t rounding = 0;       // 0: exact half-to-even; 1: rint(t * k) with k = (m_i - 1)/(m - 1) in fp64
};

// The rounding rule for merge tables, set from PlanConfig::rounding while a
// plan is built (plan building is single-threaded per call).
void set_rounding_rule(int32_t rule);

struct HostPlan {
  PlanConfig cfg;
  int32_t in_size = 1, acc_size = 4;
  QuadDesc quad[4];
  int32_t nquad = 0;                 // number of requested quadrants
  int32_t quad_id[4];                // quadrant index of slot k
  int64_t ws_quad_off[4];            // element offset of each quadrant's buffers in the workspace
  int32_t ws_pitch[4];               // row pitch of each quadrant's buffers (elements)
  int32_t nbuf[4];
  int64_t out_elems = 0;
  size_t ws_bytes = 0;               // includes the 256-byte status header
  std::vector<FusedItem> fused;
  std::vector<MergeOp> ops;
  std::vector<RowJob> rows;          // all upper passes, pass after pass
  std::vector<int64_t> pass_begin;   // rows[pass_begin[p] .. pass_begin[p+1])
  std::vector<int64_t> pass_bytes;   // model bytes of each upper pass
  int64_t fused_bytes = 0;           // model bytes of the fused pass
  // adjoint
  std::vector<AdjRow> arows;         // all adjoint upper passes, highest first
  std::vector<AdjTerm> aterms;
  std::vector<int64_t> apass_begin;  // arows[apass_begin[p] .. apass_begin[p+1])
  std::vector<int32_t> aptr;         // fused adjoint programs: CSR row pointers into aops
  std::vector<MergeOp> aops;         // (top = forward dst row r, s = shift): g[k][j] += g'[r][j - s]
  size_t adj_ws_bytes = 0;
  bool has_adjoint = false;          // adjoint tables built (cfg.with_adjoint)
  int32_t upper_heights = 0;         // tree heights above the fused subtrees (per-height passes)
  int32_t max_antiles = 0;
  int32_t max_ntiles = 0;
  int32_t max_fused_m = 1;
  int32_t max_fused_shift = 0;        // largest shift s of any fused merge
  int32_t max_generic_m = 0;          // tallest subtree on the generic fused path (0: none)
  int32_t generic_shift = 0;          // largest shift of a generic fused merge
  int32_t generic_tw = 0;             // column tile of generic fused items
  int32_t n_by64 = 0;                 // fused items on the 64-row Brady-Yong fast path
  // register-tiled block path (4-byte accumulators, tile kVTile, kVThreads
  // threads): the 64-row blocks run in a launch of their own, after one for
  // the generic subtrees (fused[0 .. n_generic) sorts first)
  bool vblock = false;
  // adjoint fused kernel: its own column tile and CTA size (the forward's
  // register-tiled shape does not suit its shared-memory radix-2 path)
  int32_t adj_tw = 0, adj_threads = 0;
  int32_t n_generic = 0;
  int32_t max_generic_ntiles = 0, max_by64_ntiles = 0;
  int64_t generic_bytes = 0, by64_bytes = 0;  // model bytes of the two kinds of fused items
  int64_t adds = 0, model_bytes = 0, ideal_bytes = 0;
  // band schedule (Split_T with 64-row fused blocks): one gathered
  // Brady-Yong pass for every perfect band above the blocks, then one
  // spine-sum pass, replacing the per-height passes
  bool bands = false;
  std::vector<FusedItem> band_items;
  std::vector<SpineRow> spine_rows;       // all spine launches, lowest chunk level first
  std::vector<SpineTerm> spine_terms;
  std::vector<int64_t> spine_pass_begin;  // spine_rows[spine_pass_begin[k] .. spine_pass_begin[k+1])
  std::vector<int64_t> spine_pass_bytes;
  // staged spine kernel: per pass, its 16-row groups (spine_grps[spine_grp_begin[k] ..]) and the
  // shared-memory elements the largest group needs (0: the pass runs the unstaged kernel)
  std::vector<SpineSeg> spine_segs;
  std::vector<SpineGrp> spine_grps;
  std::vector<int64_t> spine_grp_begin;
  std::vector<int32_t> spine_pass_smem;
  int32_t max_band_ntiles = 0;
  int64_t band_bytes = 0, spine_bytes = 0;
  int32_t max_spine_terms = 0;
};

// Returns "" on success, else an error message.
std::string build_plan(const PlanConfig& cfg, HostPlan& out);

// Verifies, on the host, that every memory access the kernels derive from the
// plan's tables stays inside its buffer (input, workspace, output, shared
// window).  Returns "" or the first violation.
struct FusedGeometry;
std::string check_plan(const HostPlan& P, const FusedGeometry& g, int32_t adj_rp, int32_t adj_padl);

// Bytes of the status header at the start of every workspace.
constexpr size_t kWsHeader = 256;

}  // namespace fht

// Host plan builder (see plan.hpp).
//
// The transform of one quadrant is Algorithm 1 of Section 3 run on the
// quadrant's view V (n rows split recursively, rows of length W).  The
// calculation-order tree G(n) of Theorem 1's proof is built once; its nodes
// are then scheduled in two kinds of passes:
//   * fused pass: every maximal subtree of at most F rows is merged in shared
//     memory from the input rows (one HBM read of the image, one write);
//   * upper passes: one pass per tree height above the fused subtrees, each a
//     gather-add over whole rows in HBM (Algorithm 1's merge, line by line).
#include "plan.hpp"

#include <algorithm>
#include <cmath>
#include <map>
#include <set>

namespace fht {

static int32_t ceil_log2(int64_t n) {
  int32_t k = 0;
  while ((int64_t(1) << k) < n) k++;
  return k;
}

void split_sizes(int32_t n, Split rule, int32_t& n0, int32_t& n1) {
  if (rule == Split::T) {
    n0 = (int32_t)(int64_t(1) << (ceil_log2(n) - 1));
  } else {
    n0 = n / 2;
  }
  n1 = n - n0;
}

int64_t round_half_even(int64_t a, int64_t d) {
  int64_t q = a / d, r = a % d;
  if (2 * r > d) return q + 1;
  if (2 * r < d) return q;
  return q + (q & 1);
}

static thread_local int32_t g_rounding = 0;

void set_rounding_rule(int32_t rule) { g_rounding = rule; }

// Algorithm 1 writes k_P = (w_P - 1)/(w - 1), then [t k_P].  Rule 1 reads it
// literally in floating point: k in double, then round-to-nearest-even of the
// product; it differs from the exact rule only where t (m_i - 1)/(m - 1) is a
// tie that the double product misses.
static inline int32_t float_k_round(int32_t t, int32_t mi, int32_t m) {
  const double k = (double)(mi - 1) / (double)(m - 1);
  return (int32_t)rint((double)t * k);
}

void merge_entry(int32_t m, int32_t m0, int32_t m1, int32_t t, int32_t& t1, int32_t& t2, int32_t& s) {
  if (g_rounding == 1) {
    t1 = float_k_round(t, m0, m);
    t2 = float_k_round(t, m1, m);
  } else {
    t1 = (int32_t)round_half_even((int64_t)t * (m0 - 1), m - 1);
    t2 = (int32_t)round_half_even((int64_t)t * (m1 - 1), m - 1);
  }
  s = t - t2;
}

// Nearest integer to q + r / d (0 <= r < d), ties to even.
static inline int32_t round_qr(int64_t q, int64_t r, int64_t d) {
  if (2 * r > d) return (int32_t)(q + 1);
  if (2 * r < d) return (int32_t)q;
  return (int32_t)(q + (q & 1));
}

void merge_table(int32_t m, int32_t m0, int32_t m1, std::vector<MergeRow>& out) {
  out.resize(m);
  if (g_rounding == 1) {
    for (int32_t t = 0; t < m; t++) {
      const int32_t t2 = float_k_round(t, m1, m);
      out[t] = MergeRow{float_k_round(t, m0, m), t2, t - t2};
    }
    return;
  }
  const int64_t d = m - 1;
  int64_t q0 = 0, r0 = 0, q1 = 0, r1 = 0;  // t (m0 - 1) = q0 d + r0, t (m1 - 1) = q1 d + r1
  for (int32_t t = 0; t < m; t++) {
    const int32_t t1 = round_qr(q0, r0, d), t2 = round_qr(q1, r1, d);
    out[t] = MergeRow{t1, t2, t - t2};
    r0 += m0 - 1;  // m_i - 1 < d, so one subtraction restores r < d
    if (r0 >= d) {
      r0 -= d;
      q0++;
    }
    r1 += m1 - 1;
    if (r1 >= d) {
      r1 -= d;
      q1++;
    }
  }
}

static int32_t build_rec(Tree& tr, int32_t a, int32_t m, Split rule) {
  TreeNode nd;
  nd.a = a;
  nd.m = m;
  if (m > 1) {
    int32_t m0, m1;
    split_sizes(m, rule, m0, m1);
    int32_t c0 = build_rec(tr, a, m0, rule);
    int32_t c1 = build_rec(tr, a + m0, m1, rule);
    nd.child[0] = c0;
    nd.child[1] = c1;
    nd.height = 1 + std::max(tr.nodes[c0].height, tr.nodes[c1].height);
  }
  tr.nodes.push_back(nd);
  return (int32_t)tr.nodes.size() - 1;
}

Tree build_tree(int32_t n, Split rule) {
  Tree tr;
  tr.n = n;
  tr.nodes.reserve(2 * (size_t)n);
  build_rec(tr, 0, n, rule);
  return tr;
}

// Program of a subtree of m rows rooted at node `r` of `tr`: for each level
// (1..height) and each local row, the merge that produces it, or a carry.
static void build_program(const Tree& tr, int32_t r, std::vector<MergeOp>& ops, int32_t& nlev) {
  const TreeNode& root = tr.nodes[r];
  nlev = root.height;
  const int32_t m = root.m, base = root.a;
  // collect the subtree's internal nodes by height (the lists and the merge
  // table are this thread's scratch, reused from one subtree to the next)
  static thread_local std::vector<std::vector<int32_t>> by_h;
  static thread_local std::vector<int32_t> stack;
  static thread_local std::vector<MergeRow> mtab;
  if ((int32_t)by_h.size() < nlev + 1) by_h.resize(nlev + 1);
  for (int32_t lev = 0; lev <= nlev; lev++) by_h[lev].clear();
  stack.assign(1, r);
  while (!stack.empty()) {
    int32_t i = stack.back();
    stack.pop_back();
    const TreeNode& nd = tr.nodes[i];
    if (nd.m > 1) {
      by_h[nd.height].push_back(i);
      stack.push_back(nd.child[0]);
      stack.push_back(nd.child[1]);
    }
  }
  for (int32_t lev = 1; lev <= nlev; lev++) {
    size_t off = ops.size();
    ops.resize(off + m);
    for (int32_t j = 0; j < m; j++) ops[off + j] = MergeOp{(int16_t)j, (int16_t)-1, 0, 0};
    for (int32_t i : by_h[lev]) {
      const TreeNode& nd = tr.nodes[i];
      const TreeNode& c0 = tr.nodes[nd.child[0]];
      const TreeNode& c1 = tr.nodes[nd.child[1]];
      merge_table(nd.m, c0.m, c1.m, mtab);
      for (int32_t t = 0; t < nd.m; t++) {
        const int32_t t1 = mtab[t].t1, t2 = mtab[t].t2, s = mtab[t].s;
        MergeOp op;
        op.top = (int16_t)(c0.a - base + t1);
        op.bot = (int16_t)(c1.a - base + t2);
        op.s = (int16_t)s;
        op.pad = 0;
        ops[off + (nd.a - base) + t] = op;
      }
    }
  }
}

// Adjoint of a fused program: for each level and each source row k, the
// forward outputs that read it, as a CSR list of (forward dst row r, shift s):
// the gradient of k at column j gathers the gradient of r at column j - s.
static void build_adjoint_program(const std::vector<MergeOp>& ops, int32_t prog, int32_t nlev, int32_t m,
                                  std::vector<int32_t>& aptr, std::vector<MergeOp>& aops, int32_t& aoff) {
  aoff = (int32_t)aptr.size();
  for (int32_t lev = 0; lev < nlev; lev++) {
    std::vector<std::vector<MergeOp>> by_src(m);
    for (int32_t r = 0; r < m; r++) {
      const MergeOp& op = ops[(size_t)prog + (size_t)lev * m + r];
      by_src[op.top].push_back(MergeOp{(int16_t)r, 0, 0, 0});
      if (op.bot >= 0) by_src[op.bot].push_back(MergeOp{(int16_t)r, 0, op.s, 0});
    }
    for (int32_t k = 0; k < m; k++) {
      aptr.push_back((int32_t)aops.size());
      for (const MergeOp& t : by_src[k]) aops.push_back(t);
    }
    aptr.push_back((int32_t)aops.size());  // end of this level's last row
  }
}

static int32_t bi_width(const PlanConfig& cfg, const QuadDesc& Q, int32_t m) {
  return cfg.ext ? Q.L + m - 1 : Q.W;
}

static int32_t dtype_in_size(int32_t dt) { return dt == 0 ? 1 : dt == 3 ? 8 : 4; }
static int32_t dtype_acc_size(int32_t dt) { return dt == 3 ? 8 : 4; }

// Segments of the staged spine kernel, pass by pass and 16-row group by
// group (the grouping of the kernel's CTAs).  Terms of one group that read
// the same part row at offsets within kStageMaxSpan of each other share one
// window [u0 + a_off, u0 + a_off + len) of that row; every term records where
// its column u0 lands in the group's shared buffer (sofs).  A pass whose
// largest group needs more than kStageSmemMax bytes, or whose cyclic rows are
// too short for the window arithmetic, keeps the unstaged kernel.
static constexpr size_t kStageSmemMax = 96 << 10;

static void build_spine_staging(HostPlan& P) {
  const int32_t acc = P.acc_size;
  const int32_t epc = 16 / acc;  // elements per 16-byte chunk
  // m is a power of two (elements per 16 bytes): round by masking
  auto floor_to = [](int64_t a, int64_t m) { return a & ~(m - 1); };
  auto ceil_to = [](int64_t a, int64_t m) { return (a + m - 1) & ~(m - 1); };
  struct Seg {
    int64_t row;
    int32_t wpart, lo, hi;
  };
  // this thread's scratch, reused by every group and every plan
  static thread_local std::vector<Seg> segs;
  static thread_local std::vector<std::pair<int64_t, int32_t>> member;  // term index -> segment
  // A group's segments of one part row are chained in index order (next[])
  // from a hash of the row (open addressing over kHash slots), so a term looks
  // only at its own row's segments and still takes the first that fits.
  constexpr int32_t kHash = 2048;
  static thread_local std::vector<int64_t> hkey(kHash);
  static thread_local std::vector<int32_t> hhead(kHash, -1), htail(kHash, -1), hused, next;
  for (int32_t s : hused) hhead[s] = -1;  // an earlier plan's last group
  hused.clear();
  P.spine_grps.reserve(P.spine_rows.size() / kSpineRows + P.spine_pass_begin.size());
  P.spine_grp_begin.push_back(0);
  for (size_t p = 0; p + 1 < P.spine_pass_begin.size(); p++) {
    const int64_t b = P.spine_pass_begin[p], e = P.spine_pass_begin[p + 1];
    int64_t need = 0;
    bool ok = true;
    for (int64_t g0 = b; g0 < e; g0 += kSpineRows) {
      const int64_t g1 = std::min<int64_t>(e, g0 + kSpineRows);
      segs.clear();
      member.clear();
      next.clear();
      for (int32_t s : hused) hhead[s] = -1;
      hused.clear();
      for (int64_t r = g0; r < g1; r++) {
        const SpineRow& R = P.spine_rows[r];
        const QuadDesc& Q = P.quad[R.q];
        if (!Q.ext && Q.W < kStageTile + 4 * kStageMaxSpan) ok = false;
        for (int32_t c = 0; c < R.term_count; c++) {
          const int64_t ti = R.term_begin + c;
          const SpineTerm& T = P.spine_terms[ti];
          int32_t slot = (int32_t)(((uint64_t)T.row * 0x9E3779B97F4A7C15ull) >> 53);  // 11 bits
          while (hhead[slot] != -1 && hkey[slot] != T.row) slot = (slot + 1) & (kHash - 1);
          int32_t k = -1;
          for (int32_t j = hhead[slot]; j != -1; j = next[j]) {
            Seg& S = segs[j];
            if (T.off >= S.hi - kStageMaxSpan && T.off <= S.lo + kStageMaxSpan) {
              S.lo = std::min(S.lo, T.off);
              S.hi = std::max(S.hi, T.off);
              k = j;
              break;
            }
          }
          if (k < 0) {
            k = (int32_t)segs.size();
            segs.push_back({T.row, T.wpart, T.off, T.off});
            next.push_back(-1);
            if (hhead[slot] == -1) {
              hkey[slot] = T.row;
              hhead[slot] = k;
              hused.push_back(slot);
            } else {
              next[htail[slot]] = k;
            }
            htail[slot] = k;
          }
          member.emplace_back(ti, k);
        }
      }
      if ((int32_t)segs.size() > kStageMaxSegs) ok = false;
      SpineGrp G;
      G.seg_begin = (int32_t)P.spine_segs.size();
      G.seg_count = (int32_t)segs.size();
      int64_t smem = 0;
      for (const Seg& S : segs) {
        SpineSeg o;
        o.row = S.row;
        o.wpart = S.wpart;
        o.a_off = (int32_t)floor_to(S.lo, epc);
        o.len = (int32_t)ceil_to((int64_t)S.hi + kStageTile - o.a_off, epc);
        o.smem = (int32_t)smem;
        smem += o.len;
        P.spine_segs.push_back(o);
      }
      for (const auto& m : member) {
        SpineTerm& T = P.spine_terms[m.first];
        const SpineSeg& o = P.spine_segs[G.seg_begin + m.second];
        T.sofs = o.smem + (T.off - o.a_off);
      }
      P.spine_grps.push_back(G);
      need = std::max(need, smem);
    }
    P.spine_grp_begin.push_back((int64_t)P.spine_grps.size());
    P.spine_pass_smem.push_back(ok && (size_t)need * acc <= kStageSmemMax ? (int32_t)need : 0);
  }
}

// Launch shape of the block passes when the caller sets none (0): the
// register-tiled path (kVTile columns, kVThreads threads) where it measured
// faster than the shared-memory radix-4 path on GB300 (4-byte accumulators,
// Split_T with 64-row blocks, every requested quadrant at least 2048 rows,
// not a power of two, whose root band would store through the column map
// element by element, and at least 512 columns); otherwise 128 columns (64
// for double) x 512 threads.
static void default_launch_shape(PlanConfig& c) {
  bool vt = dtype_acc_size(c.dtype) == 4 && c.split == Split::T && c.F == 64;
  for (int q = 0; q < 4; q++) {
    if (!(c.quads & (1u << q))) continue;
    const int32_t n = q < 2 ? c.h : c.w, L = q < 2 ? c.w : c.h;
    vt = vt && n >= 2048 && (n & (n - 1)) != 0 && L >= 512;
  }
  if (c.TW == 0) c.TW = vt ? kVTile : (c.dtype == 3 ? 64 : 128);
  if (c.threads == 0) c.threads = c.TW == kVTile ? kVThreads : 512;
}

std::string build_plan(const PlanConfig& cfg_in, HostPlan& P) {
  PlanConfig cfg = cfg_in;
  default_launch_shape(cfg);
  if (cfg.h < 1 || cfg.w < 1 || cfg.h > 65535 || cfg.w > 65535) return "h and w must be in [1, 65535]";
  if (cfg.dtype < 0 || cfg.dtype > 3) return "unknown dtype";
  if (cfg.quads == 0 || (cfg.quads & ~15u)) return "quadrants must be a non-empty subset of FHT_QALL";
  if (cfg.ext != 0 && cfg.ext != 1) return "unknown boundary";
  if (cfg.F < 1 || cfg.F > 64 || (cfg.F & (cfg.F - 1))) return "fused_rows must be a power of two in [1, 64]";
  if (cfg.TW < 32 || cfg.TW % 32 || cfg.TW > 1024) return "tile_cols must be a multiple of 32 in [32, 1024]";
  if (cfg.threads < 32 || cfg.threads % 32 || cfg.threads > 1024) return "threads must be a multiple of 32";
  if (cfg.generic_cols < 0 || cfg.generic_cols % 32 || cfg.generic_cols > 1024)
    return "generic_cols must be 0 or a multiple of 32 in [32, 1024]";
  if (cfg.rounding != 0 && cfg.rounding != 1) return "unknown rounding rule";
  set_rounding_rule(cfg.rounding);
  P = HostPlan();
  P.cfg = cfg;
  P.adj_tw = cfg.TW == kVTile ? 128 : cfg.TW;
  P.adj_threads = cfg.TW == kVTile ? 512 : cfg.threads;
  P.in_size = dtype_in_size(cfg.dtype);
  P.acc_size = dtype_acc_size(cfg.dtype);
  const int32_t acc = P.acc_size;

  Tree trees[2];
  bool have[2] = {false, false};
  for (int q = 0; q < 4; q++) {
    if (!(cfg.quads & (1u << q))) continue;
    int ti = q < 2 ? 0 : 1;
    if (!have[ti]) {
      trees[ti] = build_tree(ti == 0 ? cfg.h : cfg.w, cfg.split);
      have[ti] = true;
    }
  }

  std::map<int32_t, std::pair<int32_t, int32_t>> prog_cache;  // fused root size -> (prog offset, nlev)
  std::map<int32_t, int32_t> aprog_cache;                       // fused root size -> adjoint ptr offset
  std::vector<std::vector<AdjRow>> apasses;                     // by height
  std::vector<std::vector<AdjTerm>> aterms_by_h;
  int64_t out_off = 0;
  int64_t ws_off = 0;  // elements of the accumulator type after the header
  std::vector<std::vector<RowJob>> passes;
  std::vector<int64_t> bytes_by_height;
  // spine rows and terms by chunk level from the bottom, and the big parts'
  // (n > 8192) pre-pass: this thread's scratch, emptied here and reused from
  // one plan to the next (a serving process builds thousands of plans a
  // second, and fresh vectors of this size cost a page fault per 4 KB)
  static thread_local std::vector<SpineRow> pre_rows;
  static thread_local std::vector<SpineTerm> pre_terms;
  static thread_local std::vector<std::vector<SpineRow>> spine_levels_rows;
  static thread_local std::vector<std::vector<SpineTerm>> spine_levels_terms;
  pre_rows.clear();
  pre_terms.clear();
  for (auto& v : spine_levels_rows) v.clear();
  for (auto& v : spine_levels_terms) v.clear();
  size_t nlevels = 0;  // levels in use this plan (the scratch may hold more, empty)
  std::vector<std::vector<MergeRow>> spine_tabs[2];  // per tree: merge tables of its spine nodes
  std::vector<int64_t> chunk_row0;  // per spine chunk: first row, width, height of each part
  std::vector<int32_t> chunk_w, chunk_m;
  int64_t pre_bytes = 0;
  std::vector<int64_t> spine_levels_bytes;
  std::set<int32_t> heights_seen;

  for (int q = 0; q < 4; q++) {
    if (!(cfg.quads & (1u << q))) continue;
    const int ti = q < 2 ? 0 : 1;
    Tree tr = trees[ti];  // per-quadrant copy: buffer assignment is per quadrant
    QuadDesc& Q = P.quad[q];
    Q.transpose = q >= 2;
    Q.flip = q & 1;
    Q.n = tr.n;
    Q.L = q < 2 ? cfg.w : cfg.h;
    Q.W = cfg.ext ? Q.L + Q.n - 1 : Q.L;
    Q.ext = cfg.ext;
    // output column X of node column u:  Q0 cyclic X = u; Q0 extended X = u - (n-1) mod W;
    // Q1 cyclic X = L-1-u; Q1 extended X = W-1-u (the view of Q1 is the column-reversed image).
    if (!Q.flip) {
      Q.sigma = 1;
      Q.kappa = cfg.ext ? -(Q.n - 1) : 0;
    } else {
      Q.sigma = -1;
      Q.kappa = cfg.ext ? Q.W - 1 : Q.L - 1;
    }
    Q.out_off = out_off;
    P.quad_id[P.nquad++] = q;
    const int64_t qsize = (int64_t)Q.n * Q.W;
    out_off += qsize;

    // workspace row pitch: widest non-root node, rounded to 128 bytes
    const int32_t rootidx = tr.root();
    int32_t widest = 1;
    for (int32_t i = 0; i < (int32_t)tr.nodes.size(); i++) {
      if (i == rootidx) continue;
      int32_t wn = cfg.ext ? Q.L + tr.nodes[i].m - 1 : Q.W;
      widest = std::max(widest, wn);
    }
    const int32_t align = 128 / acc;
    const int32_t pitch = (widest + align - 1) / align * align;

    // fused roots: maximal subtrees with m <= F
    std::vector<char> is_upper(tr.nodes.size(), 0);
    std::vector<int32_t> fused_roots;
    for (int32_t i = 0; i < (int32_t)tr.nodes.size(); i++) is_upper[i] = tr.nodes[i].m > cfg.F;
    for (int32_t i = 0; i < (int32_t)tr.nodes.size(); i++) {
      const TreeNode& nd = tr.nodes[i];
      if (nd.m > cfg.F) {
        for (int c = 0; c < 2; c++)
          if (!is_upper[nd.child[c]]) fused_roots.push_back(nd.child[c]);
      }
    }
    if (!is_upper[rootidx]) fused_roots.push_back(rootidx);

    // buffer assignment: fused roots -> 0; upper nodes -> smallest buffer not used by a child
    int32_t nbuf = 1;
    for (int32_t i : fused_roots) tr.nodes[i].buf = 0;
    for (int32_t i = 0; i < (int32_t)tr.nodes.size(); i++) {
      TreeNode& nd = tr.nodes[i];
      if (!is_upper[i]) continue;
      if (i == rootidx) {
        nd.buf = -1;
        continue;
      }
      int32_t b0 = tr.nodes[nd.child[0]].buf, b1 = tr.nodes[nd.child[1]].buf;
      int32_t b = 0;
      while (b == b0 || b == b1) b++;
      nd.buf = b;
      nbuf = std::max(nbuf, b + 1);
    }
    const bool root_fused = !is_upper[rootidx];
    if (root_fused) nbuf = 0;  // the single fused subtree writes the output directly
    // band schedule: walk the Split_T spine from the root; every left child is
    // a power of two, the walk ends at a power of two or at the remainder
    // subtree of at most 64 rows.  A power of two of at most 4096 rows is a
    // part (a perfect band of 64-row blocks, or one block); a larger one (n >
    // 8192) is a "big" part, summed in a pre-pass from its 4096-row bands.
    const bool use_bands = cfg.split == Split::T && cfg.F == 64 && !root_fused;
    std::vector<int32_t> spine, parts, bands, big;
    // spine chunks of spine_chunk consecutive spine nodes, from the bottom:
    // [k_top, k_bottom] indices into `spine`.  The top node of every chunk but
    // the highest is an inner node, summed first into its own compact rows
    // after the buffers, and a single part of the chunk above.  Big parts
    // live in the same compact region.
    std::vector<std::pair<int32_t, int32_t>> chunks;
    std::vector<int64_t> inner_row0_of(tr.nodes.size(), -1);  // first compact row of an inner or big node
    int64_t inner_rows = 0;
    auto is_pow2 = [&](int32_t i) { return (tr.nodes[i].m & (tr.nodes[i].m - 1)) == 0; };
    auto is_part = [&](int32_t i) { return tr.nodes[i].m <= 64 || (is_pow2(i) && tr.nodes[i].m <= kMaxBandRows); };
    if (use_bands) {
      int32_t i = rootidx;
      while (!is_part(i)) {
        spine.push_back(i);
        parts.push_back(tr.nodes[i].child[0]);
        i = tr.nodes[i].child[1];
      }
      parts.push_back(i);
      // the bands: parts of 128..4096 rows, and the 4096-row bands under big parts
      for (int32_t pi : parts) {
        if (is_part(pi)) {
          if (tr.nodes[pi].m > 64) bands.push_back(pi);
          continue;
        }
        big.push_back(pi);
        std::vector<int32_t> stack{pi};
        while (!stack.empty()) {
          const int32_t v = stack.back();
          stack.pop_back();
          if (tr.nodes[v].m <= kMaxBandRows) {
            bands.push_back(v);
          } else {
            stack.push_back(tr.nodes[v].child[1]);
            stack.push_back(tr.nodes[v].child[0]);
          }
        }
      }
      for (int32_t bi : bands)
        if (bi != rootidx) nbuf = std::max(nbuf, 2);
      for (int32_t bi : big) {
        inner_row0_of[bi] = inner_rows;
        inner_rows += tr.nodes[bi].m;
      }
      const int32_t C = std::max(1, cfg.spine_chunk);
      for (int32_t kb = (int32_t)spine.size() - 1; kb >= 0; kb -= C) chunks.emplace_back(std::max(0, kb - C + 1), kb);
      for (size_t c = 0; c + 1 < chunks.size(); c++) {
        inner_row0_of[spine[chunks[c].first]] = inner_rows;
        inner_rows += tr.nodes[spine[chunks[c].first]].m;
      }
      P.bands = true;
    }
    P.ws_quad_off[q] = ws_off;
    P.ws_pitch[q] = pitch;
    P.nbuf[q] = nbuf;
    const int64_t bufsize = (int64_t)tr.n * pitch;
    ws_off += nbuf * bufsize + inner_rows * pitch;
    const int64_t inner_base = P.ws_quad_off[q] + nbuf * bufsize;
    auto buf_row = [&](int32_t b, int32_t row) -> int64_t {
      return P.ws_quad_off[q] + (int64_t)b * bufsize + (int64_t)row * pitch;
    };

    // fused items
    for (int32_t i : fused_roots) {
      const TreeNode& nd = tr.nodes[i];
      auto it = prog_cache.find(nd.m);
      if (it == prog_cache.end()) {
        int32_t off = (int32_t)P.ops.size(), nlev = 0;
        build_program(tr, i, P.ops, nlev);
        it = prog_cache.emplace(nd.m, std::make_pair(off, nlev)).first;
      }
      FusedItem fi{};
      fi.aprog = -1;
      if (cfg.with_adjoint) {
        auto ait = aprog_cache.find(nd.m);
        if (ait == aprog_cache.end()) {
          int32_t aoff = 0;
          build_adjoint_program(P.ops, it->second.first, it->second.second, nd.m, P.aptr, P.aops, aoff);
          ait = aprog_cache.emplace(nd.m, aoff).first;
        }
        fi.aprog = ait->second;
      }
      fi.antiles = (Q.L + P.adj_tw - 1) / P.adj_tw;
      P.max_antiles = std::max(P.max_antiles, fi.antiles);
      fi.q = q;
      fi.a = nd.a;
      fi.m = nd.m;
      fi.prog = it->second.first;
      fi.nlev = it->second.second;
      fi.wn = cfg.ext ? Q.L + nd.m - 1 : Q.W;
      fi.c = cfg.ext ? nd.m - 1 : 0;
      fi.final_ = (i == rootidx);
      if (fi.final_) {
        fi.dst = Q.out_off;
        fi.dst_pitch = Q.W;
      } else {
        fi.dst = buf_row(nd.buf, nd.a);
        fi.dst_pitch = pitch;
      }
      // a 64-row subtree is a perfect Brady-Yong block under both split rules
      fi.kind = nd.m == 64 ? FUSED_BY64 : FUSED_GENERIC;
      fi.L = fi.kind == FUSED_BY64 ? 6 : 0;
      fi.tw = 0;  // set once all items are known
      fi.ntiles = 0;
      P.max_fused_m = std::max(P.max_fused_m, nd.m);
      P.fused.push_back(fi);
      // model bytes: the subtree's input rows once, its Hough rows once
      P.fused_bytes += (int64_t)nd.m * Q.L * P.in_size + (int64_t)nd.m * fi.wn * acc;
    }

    if (use_bands) {
      // part p of the spine lives in buffer 0 (<= 64 rows: written by the fused
      // pass) or buffer 1 (a band: written by the band pass), or is the root
      auto part_buf = [&](int32_t pi) { return tr.nodes[pi].m <= 64 ? 0 : 1; };
      auto part_w = [&](int32_t pi) { return cfg.ext ? Q.L + tr.nodes[pi].m - 1 : Q.W; };
      for (int32_t pi : bands) {
        const TreeNode& band = tr.nodes[pi];
        const bool fin = pi == rootidx;
        const int32_t B = band.m / 64, G = 64 / B;
        int32_t L = 0;
        while ((1 << L) < B) L++;
        for (int32_t K0 = 0; K0 < 64; K0 += G) {
          FusedItem bi{};
          bi.q = q;
          bi.kind = FUSED_BAND;
          bi.a = band.a;
          bi.m = 64;
          bi.L = L;
          bi.B = B;
          bi.K0 = K0;
          bi.src = buf_row(0, band.a);
          bi.src_pitch = pitch;
          bi.wsrc = cfg.ext ? Q.L + 63 : Q.W;
          bi.c_src = cfg.ext ? 63 : 0;
          bi.wn = part_w(pi);
          bi.c = cfg.ext ? band.m - 1 : 0;
          bi.final_ = fin;
          bi.dst = fin ? Q.out_off + (int64_t)K0 * B * Q.W : buf_row(1, band.a + K0 * B);
          bi.dst_pitch = fin ? Q.W : pitch;
          bi.tw = cfg.TW;
          bi.ntiles = (bi.wn + bi.tw - 1) / bi.tw;
          P.max_band_ntiles = std::max(P.max_band_ntiles, bi.ntiles);
          P.band_items.push_back(bi);
        }
        // compulsory bytes: the band's blocks read once, the band written once
        P.band_bytes += ((int64_t)band.m * (cfg.ext ? Q.L + 63 : Q.W) + (int64_t)band.m * bi_width(cfg, Q, band.m)) * acc;
      }
      if (!spine.empty()) {
        // the spine nodes' merge tables, once per tree (Q0 / Q1 and Q2 / Q3 share theirs)
        std::vector<std::vector<MergeRow>>& stab = spine_tabs[ti];
        if (stab.empty()) {
          stab.resize(spine.size());
          for (size_t k = 0; k < spine.size(); k++) {
            const TreeNode& nd = tr.nodes[spine[k]];
            merge_table(nd.m, tr.nodes[nd.child[0]].m, tr.nodes[nd.child[1]].m, stab[k]);
          }
        }
        auto node_row = [&](int32_t pi, int32_t row) -> int64_t {
          if (inner_row0_of[pi] >= 0) return inner_base + (inner_row0_of[pi] + row) * pitch;
          return buf_row(part_buf(pi), tr.nodes[pi].a + row);
        };
        auto node_w = [&](int32_t pi) { return cfg.ext ? Q.L + tr.nodes[pi].m - 1 : Q.W; };
        // pre-pass: every big part, as the sum over its 4096-row bands; the
        // terms follow the merges of its subtree, t -> (t1, t2, s), down to
        // the bands, accumulating the shifts
        for (int32_t bi : big) {
          const TreeNode& N = tr.nodes[bi];
          for (int32_t t = 0; t < N.m; t++) {
            SpineRow sr{};
            sr.dst = node_row(bi, t);
            sr.q = q;
            sr.flags = SPINE_INNER;
            sr.w = node_w(bi);
            sr.term_begin = (int32_t)pre_terms.size();
            struct Visit {
              int32_t v, t;
              int64_t off;
            };
            std::vector<Visit> stack{{bi, t, 0}};
            while (!stack.empty()) {
              const Visit z = stack.back();
              stack.pop_back();
              const TreeNode& nd = tr.nodes[z.v];
              if (nd.m <= kMaxBandRows) {
                SpineTerm st{};
                st.row = node_row(z.v, z.t);
                st.wpart = node_w(z.v);
                st.off = cfg.ext ? (int32_t)(z.off + nd.m - N.m) : (int32_t)z.off;
                pre_terms.push_back(st);
                continue;
              }
              int32_t t1, t2, sh;
              merge_entry(nd.m, tr.nodes[nd.child[0]].m, tr.nodes[nd.child[1]].m, z.t, t1, t2, sh);
              int64_t off2 = z.off + sh;
              if (!cfg.ext && off2 >= Q.W) off2 %= Q.W;
              stack.push_back({nd.child[1], t2, off2});
              stack.push_back({nd.child[0], t1, z.off});
            }
            sr.term_count = (int32_t)pre_terms.size() - sr.term_begin;
            P.max_spine_terms = std::max(P.max_spine_terms, sr.term_count);
            pre_rows.push_back(sr);
          }
          // compulsory bytes: the bands once, the big part written once
          pre_bytes += 2 * (int64_t)N.m * node_w(bi) * acc;
        }
        if ((int32_t)spine_levels_rows.size() < (int32_t)chunks.size()) spine_levels_rows.resize(chunks.size());
        if ((int32_t)spine_levels_terms.size() < (int32_t)chunks.size()) spine_levels_terms.resize(chunks.size());
        if ((int32_t)spine_levels_bytes.size() < (int32_t)chunks.size()) spine_levels_bytes.resize(chunks.size(), 0);
        nlevels = std::max(nlevels, chunks.size());
        for (size_t c = 0; c < chunks.size(); c++) {
          const int32_t ktop = chunks[c].first, kbot = chunks[c].second;
          const int32_t top = spine[ktop];
          const TreeNode& N = tr.nodes[top];
          const bool fin = top == rootidx;
          std::vector<SpineRow>& rows_out = spine_levels_rows[c];
          std::vector<SpineTerm>& terms_out = spine_levels_terms[c];
          // every slope t of the chunk's top node: follow the spine down to the
          // chunk's lower boundary, collecting (part, row, offset).  A part's
          // row r lives at node_row(pi, 0) + r * pitch; its first row, width
          // and height are taken once per chunk.
          const int32_t nk = kbot - ktop + 2;  // the chunk's left parts, then its lowest node
          chunk_row0.resize(nk);
          chunk_w.resize(nk);
          chunk_m.resize(nk);
          for (int32_t j = 0; j < nk; j++) {
            const int32_t pi = j + 1 < nk ? tr.nodes[spine[ktop + j]].child[0] : tr.nodes[spine[kbot]].child[1];
            chunk_row0[j] = node_row(pi, 0);
            chunk_w[j] = node_w(pi);
            chunk_m[j] = tr.nodes[pi].m;
          }
          rows_out.reserve(rows_out.size() + N.m);
          terms_out.reserve(terms_out.size() + (size_t)N.m * nk);
          for (int32_t t = 0; t < N.m; t++) {
            SpineRow sr{};
            sr.dst = fin ? Q.out_off + (int64_t)t * Q.W : node_row(top, t);
            sr.q = q;
            sr.flags = fin ? 0 : SPINE_INNER;
            sr.w = fin ? Q.W : node_w(top);
            sr.term_begin = (int32_t)terms_out.size();  // rebased when the launches are flattened
            int32_t tn = t;
            int64_t off = 0;  // accumulated shift in window (x) coordinates
            auto add_term = [&](int32_t j, int32_t row) {
              SpineTerm st{};
              st.row = chunk_row0[j] + (int64_t)row * pitch;
              st.wpart = chunk_w[j];
              st.off = cfg.ext ? (int32_t)(off + chunk_m[j] - N.m) : (int32_t)off;  // off kept reduced mod W
              terms_out.push_back(st);
            };
            for (int32_t k = ktop; k <= kbot; k++) {
              const MergeRow& mr = stab[k][tn];
              add_term(k - ktop, mr.t1);
              off += mr.s;
              if (!cfg.ext && off >= Q.W) off = off < 2 * (int64_t)Q.W ? off - Q.W : off % Q.W;
              tn = mr.t2;
              if (k == kbot) add_term(nk - 1, mr.t2);
            }
            sr.term_count = (int32_t)terms_out.size() - sr.term_begin;
            P.max_spine_terms = std::max(P.max_spine_terms, sr.term_count);
            rows_out.push_back(sr);
          }
          // compulsory bytes of this launch: its parts once, its node written once
          int64_t by = (int64_t)N.m * (fin ? Q.W : node_w(top));
          for (int32_t k = ktop; k <= kbot; k++) {
            const int32_t pi = tr.nodes[spine[k]].child[0];
            by += (int64_t)tr.nodes[pi].m * node_w(pi);
          }
          const int32_t low = tr.nodes[spine[kbot]].child[1];
          by += (int64_t)tr.nodes[low].m * node_w(low);
          spine_levels_bytes[c] += by * acc;
        }
      }
    }

    // upper passes: one per tree height, shared by all quadrants
    for (int32_t i = 0; i < (int32_t)tr.nodes.size(); i++) {
      const TreeNode& nd = tr.nodes[i];
      if (!is_upper[i]) continue;
      const TreeNode& c0 = tr.nodes[nd.child[0]];
      const TreeNode& c1 = tr.nodes[nd.child[1]];
      if ((int32_t)passes.size() <= nd.height) {
        passes.resize(nd.height + 1);
        bytes_by_height.resize(nd.height + 1, 0);
      }
      heights_seen.insert(nd.height);
      const bool fin = (i == rootidx);
      const int32_t wout = cfg.ext ? Q.L + nd.m - 1 : Q.W;
      const int32_t wtop = cfg.ext ? Q.L + c0.m - 1 : Q.W;
      const int32_t wbot = cfg.ext ? Q.L + c1.m - 1 : Q.W;
      std::vector<MergeRow> mtab;
      if (!use_bands || cfg.with_adjoint) merge_table(nd.m, c0.m, c1.m, mtab);
      // per-height forward rows: only for trees that do not use the band schedule
      for (int32_t t = 0; t < (use_bands ? 0 : nd.m); t++) {
        const int32_t t1 = mtab[t].t1, t2 = mtab[t].t2, s = mtab[t].s;
        RowJob rj;
        rj.dst = fin ? Q.out_off + (int64_t)t * Q.W : buf_row(nd.buf, nd.a + t);
        rj.top = buf_row(c0.buf, c0.a + t1);
        rj.bot = buf_row(c1.buf, c1.a + t2);
        rj.wout = wout;
        rj.wtop = wtop;
        rj.wbot = wbot;
        if (cfg.ext) {
          rj.dtop = -c1.m;
          rj.dbot = s - c0.m;
        } else {
          rj.dtop = 0;
          rj.dbot = (int32_t)(s % Q.W);
        }
        rj.W = Q.W;
        rj.flags = (fin ? ROW_FINAL : 0) | (cfg.ext ? ROW_EXT : 0) | (Q.sigma < 0 ? ROW_NEG : 0);
        rj.kappa = Q.kappa;
        passes[nd.height].push_back(rj);
      }
      bytes_by_height[nd.height] += ((int64_t)c0.m * wtop + (int64_t)c1.m * wbot + (int64_t)nd.m * wout) * acc;
      // adjoint: each child row gathers the parent rows that read it
      if (!cfg.with_adjoint) continue;
      if ((int32_t)apasses.size() <= nd.height) {
        apasses.resize(nd.height + 1);
        aterms_by_h.resize(nd.height + 1);
      }
      for (int c = 0; c < 2; c++) {
        const TreeNode& ch = c == 0 ? c0 : c1;
        std::vector<std::vector<AdjTerm>> lists(ch.m);
        for (int32_t t = 0; t < nd.m; t++) {
          const int32_t t1 = mtab[t].t1, t2 = mtab[t].t2, s = mtab[t].s;
          int32_t e;
          if (c == 0) {
            e = cfg.ext ? c1.m : 0;  // -dtop
          } else {
            e = cfg.ext ? c0.m - s : (int32_t)(((int64_t)Q.W - s % Q.W) % Q.W);  // -dbot
          }
          lists[c == 0 ? t1 : t2].push_back(AdjTerm{t, e});
        }
        for (int32_t r = 0; r < ch.m; r++) {
          AdjRow ar;
          ar.dst = buf_row(ch.buf, ch.a + r);
          ar.src = fin ? Q.out_off : buf_row(nd.buf, nd.a);
          ar.src_pitch = fin ? Q.W : pitch;
          ar.wdst = c == 0 ? wtop : wbot;
          ar.wsrc = wout;
          ar.W = Q.W;
          ar.flags = (fin ? ROW_FINAL : 0) | (cfg.ext ? ROW_EXT : 0) | (Q.sigma < 0 ? ROW_NEG : 0);
          ar.kappa = Q.kappa;
          ar.term_begin = (int32_t)aterms_by_h[nd.height].size();  // rebased when passes are flattened
          ar.term_count = (int32_t)lists[r].size();
          for (const AdjTerm& at : lists[r]) aterms_by_h[nd.height].push_back(at);
          apasses[nd.height].push_back(ar);
        }
      }
    }
    // additions (Theorem 1): every merged element of every internal node is one addition
    for (const TreeNode& nd : tr.nodes)
      if (nd.m > 1) P.adds += (int64_t)nd.m * (cfg.ext ? Q.L + nd.m - 1 : Q.W);
    P.ideal_bytes += (int64_t)Q.n * Q.L * P.in_size + qsize * acc;
  }
  // spine launches: the big parts, then the lowest chunk level of every quadrant first
  P.spine_pass_begin.push_back(0);
  {
    size_t nrows = pre_rows.size(), nterms = pre_terms.size();
    for (size_t c = 0; c < nlevels; c++) {
      nrows += spine_levels_rows[c].size();
      nterms += spine_levels_terms[c].size();
    }
    P.spine_rows.reserve(nrows);
    P.spine_terms.reserve(nterms);
  }
  auto flatten = [&](const std::vector<SpineRow>& rows, const std::vector<SpineTerm>& terms, int64_t bytes) {
    const int32_t base = (int32_t)P.spine_terms.size();
    for (SpineRow sr : rows) {
      sr.term_begin += base;
      P.spine_rows.push_back(sr);
    }
    P.spine_terms.insert(P.spine_terms.end(), terms.begin(), terms.end());
    P.spine_pass_begin.push_back((int64_t)P.spine_rows.size());
    P.spine_pass_bytes.push_back(bytes);
    P.spine_bytes += bytes;
  };
  if (!pre_rows.empty()) flatten(pre_rows, pre_terms, pre_bytes);
  for (size_t c = 0; c < nlevels; c++) flatten(spine_levels_rows[c], spine_levels_terms[c], spine_levels_bytes[c]);
  build_spine_staging(P);
  // tiles: fast-path items use tile_cols; generic items (two ping-pong
  // buffers of up to 63 rows) use half of it, so their shared windows stay
  // no larger than the fast path's
  for (const FusedItem& fi : P.fused) P.n_by64 += fi.kind == FUSED_BY64;
  // generic subtrees: half the block tile by default; with the register-tiled
  // shape (their own launch, overlapping the blocks') 128 columns measured best
  // at 4095^2 (0.563 ms per step against 0.575 ms with 96 and 0.568 with 256)
  P.generic_tw = cfg.generic_cols > 0 ? cfg.generic_cols
                                      : cfg.TW == kVTile ? 128 : std::max(32, cfg.TW / 64 * 32);
  for (FusedItem& fi : P.fused) {
    fi.tw = fi.kind == FUSED_BY64 ? cfg.TW : P.generic_tw;
    fi.ntiles = (fi.wn + fi.tw - 1) / fi.tw;
    P.max_ntiles = std::max(P.max_ntiles, fi.ntiles);
    if (fi.kind == FUSED_GENERIC) {
      P.max_generic_m = std::max(P.max_generic_m, fi.m);
      for (int32_t l = 0; l < fi.nlev; l++)
        for (int32_t r = 0; r < fi.m; r++) {
          const MergeOp& op = P.ops[(size_t)fi.prog + (size_t)l * fi.m + r];
          if (op.bot >= 0) P.generic_shift = std::max<int32_t>(P.generic_shift, op.s);
        }
    }
  }
  // generic items first: they are few and slower, so they start in the first wave
  std::stable_sort(P.fused.begin(), P.fused.end(),
                   [](const FusedItem& x, const FusedItem& y) { return x.kind < y.kind; });
  for (const FusedItem& fi : P.fused) {
    const int64_t b = (int64_t)fi.m * P.quad[fi.q].L * P.in_size + (int64_t)fi.m * fi.wn * P.acc_size;
    if (fi.kind == FUSED_GENERIC) {
      P.n_generic++;
      P.max_generic_ntiles = std::max(P.max_generic_ntiles, fi.ntiles);
      P.generic_bytes += b;
    } else {
      P.max_by64_ntiles = std::max(P.max_by64_ntiles, fi.ntiles);
      P.by64_bytes += b;
    }
  }
  P.vblock = P.acc_size == 4 && cfg.TW == kVTile && cfg.threads == kVThreads && P.n_by64 > 0;

  P.out_elems = out_off;
  P.ws_bytes = kWsHeader + (size_t)ws_off * acc;
  // adjoint: one view gradient per quadrant (n rows of grad_pitch(L)) after
  // the forward buffers, each starting 16-byte aligned
  int64_t goff = (ws_off + 3) & ~(int64_t)3;
  for (int q = 0; q < 4; q++) {
    if (!(cfg.quads & (1u << q))) continue;
    P.quad[q].grad_off = goff;
    goff += (int64_t)P.quad[q].n * grad_pitch(P.quad[q].L);
  }
  P.adj_ws_bytes = kWsHeader + (size_t)goff * acc;
  // adjoint passes: highest tree height first
  P.apass_begin.push_back(0);
  for (size_t k = apasses.size(); k-- > 0;) {
    if (apasses[k].empty()) continue;
    const int32_t base = (int32_t)P.aterms.size();
    for (AdjRow ar : apasses[k]) {
      ar.term_begin += base;
      P.arows.push_back(ar);
    }
    P.aterms.insert(P.aterms.end(), aterms_by_h[k].begin(), aterms_by_h[k].end());
    P.apass_begin.push_back((int64_t)P.arows.size());
  }
  P.has_adjoint = cfg.with_adjoint;
  P.upper_heights = (int32_t)heights_seen.size();
  if (P.aterms.empty()) P.aterms.push_back(AdjTerm{0, 0});
  if (P.aops.empty()) P.aops.push_back(MergeOp{0, 0, 0, 0});
  if (P.aptr.empty()) P.aptr.push_back(0);
  // flatten passes (skip empty heights)
  P.pass_begin.push_back(0);
  P.model_bytes = P.fused_bytes;
  for (size_t k = 0; k < passes.size(); k++) {
    if (passes[k].empty()) continue;
    P.rows.insert(P.rows.end(), passes[k].begin(), passes[k].end());
    P.pass_begin.push_back((int64_t)P.rows.size());
    P.pass_bytes.push_back(bytes_by_height[k]);
    if (!P.bands) P.model_bytes += bytes_by_height[k];
  }
  if (P.bands) P.model_bytes += P.band_bytes + P.spine_bytes;
  if (P.ops.empty()) P.ops.push_back(MergeOp{0, -1, 0, 0});
  for (const MergeOp& op : P.ops)
    if (op.bot >= 0) P.max_fused_shift = std::max<int32_t>(P.max_fused_shift, op.s);
  return "";
}

}  // namespace fht

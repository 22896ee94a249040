// Descriptors shared by the host plan builder and the CUDA kernels.
// Plain structs, identical layout on host and device.
#pragma once
#include <stdint.h>

namespace fht {

// One slope quadrant of the plan.  The quadrant's "view" V is the image
// (q = 0, 1) or its transpose (q = 2, 3), with the columns reversed for the
// leftward quadrants (q = 1, 3).  Every kernel runs the rightward recursion on
// V; only the final store maps a node column u to the output column
//   X = (sigma * u + kappa) mod W.
struct QuadDesc {
  int32_t transpose;  // V[i][j] = I[j][i]
  int32_t flip;       // V[i][j] = I'[i][L - 1 - j]
  int32_t n;          // rows of V (split axis)
  int32_t L;          // real row length of V
  int32_t W;          // output row length (L, or L + n - 1 when extended)
  int32_t ext;        // extended boundary: zero outside [0, L), no wrap
  int32_t sigma;      // +1 or -1
  int32_t kappa;      // see above
  int64_t out_off;    // element offset of the quadrant in the output
  int64_t grad_off;   // adjoint: workspace offset of this quadrant's view gradient, n rows of
                      // grad_pitch(L) elements (columns [L, grad_pitch(L)) are slack)
};

// Row pitch of a quadrant's view gradient: L rounded up to 4 elements, so that
// every row starts 16-byte aligned for 4-byte accumulators.
#if defined(__CUDACC__)
__host__ __device__
#endif
inline int32_t grad_pitch(int32_t L) { return (L + 3) & ~3; }

// A subtree of at most F rows, merged entirely in shared memory.
struct FusedItem {
  int32_t q;          // quadrant
  int32_t a;          // first row of the subtree in V
  int32_t m;          // rows of the subtree
  int32_t nlev;       // merge levels (the subtree's height)
  int32_t prog;       // first MergeOp of its program: ops[prog + lev * m + r]
  int32_t wn;         // output columns of the subtree (node width)
  int32_t c;          // node column u = window column x + c
  int32_t final_;     // 1: the subtree is the whole tree, store into the output
  int64_t dst;        // element offset of its first row (workspace, or output if final_)
  int32_t dst_pitch;  // elements between rows of dst
  int32_t ntiles;     // column tiles of width tile_cols covering wn
  int32_t aprog;      // adjoint program: first row pointer (nlev * (m + 1) entries)
  int32_t antiles;    // adjoint column tiles of width tile_cols covering the view length L
  int32_t kind;       // FUSED_GENERIC, FUSED_BY64 or FUSED_BAND
  int32_t tw;         // column tile of this item (forward)
  // Brady-Yong block paths (BY64 and BAND): 64 shared rows = G groups of
  // B = 2^L rows, each group merged into a B-row Brady-Yong block.
  int32_t L;          // levels per group (6 for BY64)
  int32_t B;          // BAND: blocks of 64 rows in the band
  int32_t K0;         // BAND: first slope index of the blocks' rows (group g reads row K0 + g)
  int32_t wsrc;       // BAND: width of a block row (columns outside are zero / wrap)
  int32_t c_src;      // BAND: block column = window column x + c_src + K b
  int32_t src_pitch;  // BAND: elements between block rows
  int64_t src;        // BAND: workspace offset of row 0 of the band's first block
};

enum : int32_t { FUSED_GENERIC = 0, FUSED_BY64 = 1, FUSED_BAND = 2 };

// Register-tiled 64-row block path (4-byte accumulators, its own launch):
// CTAs of kVThreads threads, column tiles of kVTile, one shared buffer of 64
// rows x kVPitch elements.  kVPitch >= kVTile + 64, a multiple of 4 with
// kVPitch / 4 odd.
constexpr int32_t kVTile = 192;
constexpr int32_t kVThreads = 256;
constexpr int32_t kVPitch = 260;

// The quadrant table passed by value to kernels.
struct QuadDescs {
  QuadDesc q[4];
};

// Kinds of forward kernel launches (fht_plan_launch_info).
enum : int32_t { LAUNCH_FUSED = 0, LAUNCH_UPPER = 1, LAUNCH_BAND = 2, LAUNCH_SPINE = 3, LAUNCH_BLOCK = 4 };

// One output row of a root whose tree is a Split_T spine over "parts"
// (perfect bands of 2^k rows, 64-row blocks and one remainder subtree):
//   H[t][u] = sum_p part_p[r_p(t)][u + off_p(t)]
// cyclic: part index mod W; extended: zero outside [0, wpart).  A row of the
// root is stored through the quadrant's column map; a row of an inner spine
// node (the top of a lower spine chunk, itself a part of the chunk above) is
// stored in its own node-local columns in the workspace.
struct SpineRow {
  int64_t dst;        // offset of the row: the output (final) or the workspace (an inner spine node)
  int32_t q;          // quadrant
  int32_t term_begin, term_count;
  int32_t flags;      // SPINE_INNER: an inner spine node, stored in its own columns (no output map)
  int32_t w;          // columns of the row
  int32_t pad;
};

enum : int32_t { SPINE_INNER = 1 };

// Tallest perfect band the band pass builds: 64 blocks of 64 rows.
constexpr int32_t kMaxBandRows = 4096;

struct SpineTerm {
  int64_t row;        // workspace offset of the part's row r_p(t)
  int32_t wpart;      // part row width
  int32_t off;        // column offset (reduced to [0, W) in the cyclic case)
  int32_t sofs;       // staged spine kernel: shared-memory element of this term's column u0
  int32_t pad;
};

// Staged spine kernel: the rows of one 16-row group read a handful of part
// rows (consecutive slopes share them), each over a window a few columns
// wider than the column tile.  The group's distinct (part row, offset range)
// pairs are its segments; a CTA copies each segment's window into shared
// memory once, then sums every term from there.
constexpr int kMaxSpineTerms = 16;      // terms of one spine row
constexpr int kSpineRows = 16;          // spine rows per CTA (a 16-row group)
constexpr int32_t kStageTile = 512;     // columns per CTA
constexpr int32_t kStageMaxSegs = 64;   // segments per 16-row group
constexpr int32_t kStageMaxSpan = 64;   // offsets merged into one segment differ by at most this

struct SpineSeg {
  int64_t row;        // workspace offset of the part row
  int32_t wpart;      // part row width (the row length W in the cyclic case)
  int32_t a_off;      // the window starts at part column u0 + a_off (a multiple of 16 bytes)
  int32_t len;        // window length (elements, a multiple of 16 bytes)
  int32_t smem;       // first shared-memory element of the window (16-byte aligned)
};

struct SpineGrp {
  int32_t seg_begin, seg_count;
};

// One row of one level of a fused program: dst row <- src[top] + src[bot] shifted by s.
// bot < 0 means the row is carried unchanged to the next level.
struct MergeOp {
  int16_t top;
  int16_t bot;
  int16_t s;
  int16_t pad;
};

// One output row of an upper (HBM-pass) merge:
//   out[u] = top[u + dtop] + bot[u + dbot],  u in [0, wout)
// cyclic: indices taken mod W (dtop = 0, 0 <= dbot < W, wout = wtop = wbot = W);
// extended: terms outside [0, wtop) / [0, wbot) are zero.
// The final merge stores out[u] at column (sigma * u + kappa) mod W of the output row.
struct RowJob {
  int64_t dst;  // element offset of the output row (workspace or output)
  int64_t top;  // element offset of the top child's row t1 (workspace)
  int64_t bot;  // element offset of the bottom child's row t2 (workspace)
  int32_t wout, wtop, wbot;
  int32_t dtop, dbot;
  int32_t W;
  int32_t flags;  // bit0: final (dst in output), bit1: extended, bit2: sigma = -1
  int32_t kappa;
};

enum : int32_t { ROW_FINAL = 1, ROW_EXT = 2, ROW_NEG = 4 };

// Adjoint of the upper merges: one child row, gathered from the parent rows
// that read it in the forward merge (a contiguous range of slopes t, because
// t -> t1 and t -> t2 are monotone):
//   dst[i] = sum_k src[t_k][i + e_k],  i in [0, wdst)
// cyclic: index taken mod W; extended: terms with i + e_k outside [0, wsrc)
// are zero.  With ROW_FINAL the parent is the root, read from the output
// gradient through the quadrant's column map  X = (sigma * u + kappa) mod W.
struct AdjRow {
  int64_t dst;        // workspace offset of the child row
  int64_t src;        // offset of the parent's row 0 (workspace, or output gradient if final)
  int32_t src_pitch;  // elements between parent rows
  int32_t wdst, wsrc, W;
  int32_t flags;      // ROW_FINAL: src is the output gradient; ROW_EXT; ROW_NEG
  int32_t kappa;
  int32_t term_begin, term_count;
};

struct AdjTerm {
  int32_t t;  // parent row
  int32_t e;  // column offset (reduced to [0, W) in the cyclic case)
};

}  // namespace fht

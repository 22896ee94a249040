// Host-side bounds and race verification of a plan (see plan.hpp).
// Every check below mirrors an index expression of the kernels in
// fht_forward.cu; a plan that passes cannot make them touch memory outside
// the input, the workspace, the output or the shared window.
#include <algorithm>
#include <cstdint>
#include <iterator>
#include <set>
#include <string>
#include <vector>

#include "fht_launch.hpp"
#include "plan.hpp"

namespace fht {

static std::string at(const char* what, int64_t i) { return std::string(what) + " #" + std::to_string(i) + ": "; }

std::string check_plan(const HostPlan& P, const FusedGeometry& g, int32_t adj_rp, int32_t adj_padl) {
  const int64_t ws_elems = (int64_t)((P.ws_bytes - kWsHeader) / P.acc_size);
  const int64_t out_elems = P.out_elems;
  const int32_t TW = P.cfg.TW;
  for (size_t k = 0; k < P.fused.size(); k++) {
    const FusedItem& it = P.fused[k];
    if (it.q < 0 || it.q > 3 || !(P.cfg.quads & (1u << it.q))) return at("fused", k) + "bad quadrant";
    if (it.kind != FUSED_GENERIC && it.kind != FUSED_BY64) return at("fused", k) + "bad kind";
    const QuadDesc& Q = P.quad[it.q];
    const int32_t img_rows = Q.transpose ? P.cfg.w : P.cfg.h;  // view rows are image rows or columns
    const int32_t img_len = Q.transpose ? P.cfg.h : P.cfg.w;
    if (Q.n != img_rows || Q.L != img_len) return at("fused", k) + "view dims disagree with the image";
    if (it.m < 1 || it.a < 0 || it.a + it.m > Q.n) return at("fused", k) + "rows outside the view";
    if (it.m > P.max_fused_m) return at("fused", k) + "subtree taller than the shared buffers";
    if (!Q.ext && it.c != 0) return at("fused", k) + "cyclic window must start at a column >= 0";
    const int32_t tw = it.tw;
    if (tw < 32 || tw % 32) return at("fused", k) + "bad tile width";
    if (it.ntiles < 1 || (int64_t)(it.ntiles - 1) * tw >= it.wn || (int64_t)it.ntiles * tw < it.wn)
      return at("fused", k) + "tile count does not cover the node width";
    if (it.ntiles > P.max_ntiles) return at("fused", k) + "more tiles than the grid";
    const int32_t TWin = tw + it.m - 1;
    if (it.prog < 0 || (size_t)it.prog + (size_t)it.nlev * it.m > P.ops.size()) return at("fused", k) + "program";
    if (it.kind == FUSED_BY64) {
      // fast path: staged window TW + 63 in S, level-2 rows TW + 60 in A,
      // level-4 rows TW + 48 back in S; reads reach +3, +12 and +48 beyond
      if (it.m != 64 || it.nlev != 6 || it.L != 6) return at("fused", k) + "fast path needs a 64-row block";
      // the compile-time variants (tile 64, 128, 256) fix the pitches at TW + 63 and TW + 61
      if (tw != TW || g.RS != TW + 63 || g.RA != TW + 61) return at("fused", k) + "fast-path pitches";
      if (tw + 63 > g.RS || tw + 60 > g.RA || (size_t)64 * (g.RS + g.RA) * P.acc_size > g.smem)
        return at("fused", k) + "fast-path buffers too small";
      if ((tw + 60 - 1) + 3 >= g.RS || (tw + 48 - 1) + 12 >= g.RA || (tw - 1) + 48 >= g.RS)
        return at("fused", k) + "fast-path shifted read beyond a shared row";
      if (P.vblock) {
        // register-tiled launch: window kVTile + 63 staged as kVTile + 64 columns of
        // kVPitch-element rows; its own grid and shared size
        if (tw != kVTile || kVTile + 64 > kVPitch) return at("fused", k) + "register-tiled tile geometry";
        if ((int64_t)k < P.n_generic || it.ntiles > P.max_by64_ntiles)
          return at("fused", k) + "64-row block outside the block launch's grid";
        if ((size_t)64 * kVPitch * P.acc_size > g.vsmem) return at("fused", k) + "block launch shared size";
      }
      // the program must be the Brady-Yong block the fast path hard-codes
      for (int32_t l = 0; l < 6; l++) {
        const int32_t b = 1 << (l + 1);
        for (int32_t r = 0; r < 64; r++) {
          const MergeOp& op = P.ops[(size_t)it.prog + (size_t)l * 64 + r];
          const int32_t base = r / b * b, t = r - base;
          if (op.top != base + t / 2 || op.bot != base + b / 2 + t / 2 || op.s != (t + 1) / 2)
            return at("fused", k) + "64-row program is not the Brady-Yong block";
        }
      }
    } else {
      if (P.vblock && ((int64_t)k >= P.n_generic || it.ntiles > P.max_generic_ntiles ||
                       (size_t)2 * g.Fm * g.RP * P.acc_size > g.gsmem))
        return at("fused", k) + "generic subtree outside its launch's grid or shared size";
      if (it.m > g.Fm) return at("fused", k) + "subtree taller than the shared buffers";
      if ((size_t)2 * g.Fm * g.RP * P.acc_size > g.smem) return at("fused", k) + "generic buffers too small";
      for (int32_t l = 0; l < it.nlev; l++)
        for (int32_t r = 0; r < it.m; r++) {
          const MergeOp& op = P.ops[(size_t)it.prog + (size_t)l * it.m + r];
          if (op.top < 0 || op.top >= it.m) return at("fused", k) + "merge reads a row outside the subtree";
          if (op.bot >= it.m) return at("fused", k) + "merge reads a row outside the subtree";
          if (op.bot >= 0 && (op.s < 0 || TWin - 1 + op.s >= g.RP))
            return at("fused", k) + "shifted read beyond the shared row";
        }
      if (TWin > g.RP) return at("fused", k) + "window wider than the shared row";
    }
    if (!it.final_) {
      if (it.wn > it.dst_pitch) return at("fused", k) + "node wider than the workspace pitch";
      if (it.dst < 0 || it.dst + (int64_t)(it.m - 1) * it.dst_pitch + it.wn > ws_elems)
        return at("fused", k) + "store outside the workspace";
    } else {
      if (it.dst_pitch != Q.W || it.wn != Q.W) return at("fused", k) + "final subtree must span the output row";
      if (it.dst < 0 || it.dst + (int64_t)it.m * Q.W > out_elems) return at("fused", k) + "store outside the output";
      for (int32_t u : {0, it.wn - 1}) {
        const int64_t X = (int64_t)Q.sigma * u + Q.kappa;
        if (X < -Q.W || X >= 2 * (int64_t)Q.W) return at("fused", k) + "column map needs more than one wrap";
      }
    }
  }
  for (size_t p = 0; p + 1 < P.pass_begin.size(); p++) {
    std::set<int64_t> written;
    for (int64_t k = P.pass_begin[p]; k < P.pass_begin[p + 1]; k++) {
      const RowJob& J = P.rows[k];
      if (!(J.flags & ROW_FINAL)) written.insert(J.dst);
    }
    for (int64_t k = P.pass_begin[p]; k < P.pass_begin[p + 1]; k++) {
      const RowJob& J = P.rows[k];
      const bool ext = J.flags & ROW_EXT, fin = J.flags & ROW_FINAL;
      if (J.wout < 1 || J.wtop < 1 || J.wbot < 1 || J.W < 1) return at("row", k) + "empty row";
      if (ext) {
        if (J.top < 0 || J.top + J.wtop > ws_elems) return at("row", k) + "top row outside the workspace";
        if (J.bot < 0 || J.bot + J.wbot > ws_elems) return at("row", k) + "bottom row outside the workspace";
      } else {
        if (J.wtop < J.wout || J.wbot != J.W || J.wout != J.W) return at("row", k) + "cyclic widths disagree";
        if (J.dbot < 0 || J.dbot >= J.W || J.dtop != 0) return at("row", k) + "cyclic shift not reduced";
        if (J.top < 0 || J.top + J.wout > ws_elems) return at("row", k) + "top row outside the workspace";
        if (J.bot < 0 || J.bot + J.W > ws_elems) return at("row", k) + "bottom row outside the workspace";
      }
      if (written.count(J.top) || written.count(J.bot)) return at("row", k) + "reads a row written in the same pass";
      if (fin) {
        if (J.wout != J.W) return at("row", k) + "final row must span the output row";
        if (J.dst < 0 || J.dst + J.W > out_elems) return at("row", k) + "store outside the output";
        for (int32_t u : {0, J.wout - 1}) {
          const int64_t X = (J.flags & ROW_NEG) ? (int64_t)J.kappa - u : (int64_t)u + J.kappa;
          if (X < -J.W || X >= 2 * (int64_t)J.W) return at("row", k) + "column map needs more than one wrap";
        }
      } else {
        if (J.dst < 0 || J.dst + J.wout > ws_elems) return at("row", k) + "store outside the workspace";
      }
    }
  }
  if (P.vblock && (size_t)64 * kVPitch * P.acc_size > g.vsmem) return "block launch: shared buffer too small";
  // ---- band schedule ----
  for (size_t k = 0; k < P.band_items.size(); k++) {
    const FusedItem& it = P.band_items[k];
    if (!P.bands || it.kind != FUSED_BAND) return at("band", k) + "not a band item";
    if (it.tw != TW || g.RS != TW + 63 || g.RA != TW + 61) return at("band", k) + "block-path pitches";
    if (it.q < 0 || it.q > 3 || !(P.cfg.quads & (1u << it.q))) return at("band", k) + "bad quadrant";
    const QuadDesc& Q = P.quad[it.q];
    if (it.B < 2 || it.B > 64 || (it.B & (it.B - 1)) || (1 << it.L) != it.B || it.m != 64)
      return at("band", k) + "band must be 2..64 blocks of 64 rows";
    if (it.K0 < 0 || it.K0 % (64 / it.B) || it.K0 + 64 / it.B > 64) return at("band", k) + "bad group range";
    if (it.tw != TW || it.tw + 63 > g.RS || it.tw + 60 > g.RA) return at("band", k) + "band buffers too small";
    if (it.ntiles < 1 || (int64_t)(it.ntiles - 1) * TW >= it.wn || (int64_t)it.ntiles * TW < it.wn ||
        it.ntiles > P.max_band_ntiles)
      return at("band", k) + "tiles do not cover the band";
    if (!Q.ext && (it.c != 0 || it.c_src != 0 || it.wsrc != Q.W)) return at("band", k) + "cyclic offsets";
    if (it.wsrc > it.src_pitch) return at("band", k) + "block row wider than its pitch";
    if (it.src < 0 || it.src + (int64_t)(64 * (it.B - 1) + 63) * it.src_pitch + it.wsrc > ws_elems)
      return at("band", k) + "block rows outside the workspace";
    if (!it.final_) {
      if (it.wn > it.dst_pitch || it.dst < 0 || it.dst + (int64_t)63 * it.dst_pitch + it.wn > ws_elems)
        return at("band", k) + "band rows outside the workspace";
    } else {
      if (it.dst_pitch != Q.W || it.wn != Q.W || it.dst < 0 || it.dst + (int64_t)64 * Q.W > out_elems)
        return at("band", k) + "final band rows outside the output";
      for (int32_t u : {0, it.wn - 1}) {
        const int64_t X = (int64_t)Q.sigma * u + Q.kappa;
        if (X < -Q.W || X >= 2 * (int64_t)Q.W) return at("band", k) + "column map needs more than one wrap";
      }
    }
  }
  if (!P.spine_rows.empty() &&
      (P.spine_pass_begin.size() != P.spine_pass_bytes.size() + 1 || P.spine_pass_begin.front() != 0 ||
       P.spine_pass_begin.back() != (int64_t)P.spine_rows.size()))
    return "spine passes do not cover the spine rows";
  // inner spine rows: written by one pass, read only by later passes
  std::set<int64_t> inner_all, inner_written;  // inner row starts: of every pass, of earlier passes
  for (const SpineRow& R : P.spine_rows)
    if (R.flags & SPINE_INNER) inner_all.insert(R.dst);
  for (size_t p = 0; p + 1 < P.spine_pass_begin.size(); p++) {
    if (P.spine_pass_begin[p + 1] < P.spine_pass_begin[p]) return "spine passes out of order";
    std::vector<std::pair<int64_t, int64_t>> wr;  // [begin, end) written by this pass
    for (int64_t k = P.spine_pass_begin[p]; k < P.spine_pass_begin[p + 1]; k++) {
      const SpineRow& R = P.spine_rows[k];
      if (R.q < 0 || R.q > 3 || !(P.cfg.quads & (1u << R.q))) return at("spine", k) + "bad quadrant";
      const QuadDesc& Q = P.quad[R.q];
      if (R.term_count < 1 || R.term_count > 16 || R.term_begin < 0 ||
          (size_t)R.term_begin + R.term_count > P.spine_terms.size())
        return at("spine", k) + "terms";
      if (R.flags & SPINE_INNER) {
        if (R.w < 1 || R.w > Q.W || (!Q.ext && R.w != Q.W)) return at("spine", k) + "inner row width";
        if (R.dst < 0 || R.dst + R.w > ws_elems) return at("spine", k) + "inner row outside the workspace";
        wr.emplace_back(R.dst, R.dst + R.w);
      } else {
        if (R.dst < 0 || R.dst + Q.W > out_elems) return at("spine", k) + "row outside the output";
        for (int32_t u : {0, Q.W - 1}) {
          const int64_t X = (int64_t)Q.sigma * u + Q.kappa;
          if (X < -Q.W || X >= 2 * (int64_t)Q.W) return at("spine", k) + "column map needs more than one wrap";
        }
      }
      for (int32_t c = 0; c < R.term_count; c++) {
        const SpineTerm& T = P.spine_terms[R.term_begin + c];
        if (Q.ext) {
          if (T.row < 0 || T.row + T.wpart > ws_elems) return at("spine", k) + "part row outside the workspace";
        } else {
          if (T.wpart != Q.W || T.off < 0 || T.off >= Q.W || T.row < 0 || T.row + Q.W > ws_elems)
            return at("spine", k) + "cyclic part row";
        }
      }
    }
    std::sort(wr.begin(), wr.end());
    for (size_t i = 1; i < wr.size(); i++)
      if (wr[i].first < wr[i - 1].second) return "spine pass " + std::to_string(p) + ": inner rows overlap";
    // no term of this pass reads a row this pass writes; a term that reads an
    // inner row reads one an earlier pass wrote
    for (int64_t k = P.spine_pass_begin[p]; k < P.spine_pass_begin[p + 1]; k++) {
      const SpineRow& R = P.spine_rows[k];
      for (int32_t c = 0; c < R.term_count; c++) {
        const SpineTerm& T = P.spine_terms[R.term_begin + c];
        const int64_t lo = T.row, hi = T.row + T.wpart;
        auto it = std::upper_bound(wr.begin(), wr.end(), std::make_pair(lo, INT64_MAX));
        if (it != wr.begin() && std::prev(it)->second > lo) return at("spine", k) + "reads a row its pass writes";
        if (it != wr.end() && it->first < hi) return at("spine", k) + "reads a row its pass writes";
        if (inner_all.count(lo) && !inner_written.count(lo)) return at("spine", k) + "reads an inner row not yet written";
      }
    }
    for (const auto& w : wr) inner_written.insert(w.first);
  }
  // staged spine kernel: windows inside the workspace and the shared buffer,
  // every term's tile inside a window of its own part row
  if (!P.spine_rows.empty() && (P.spine_pass_smem.size() + 1 != P.spine_pass_begin.size() ||
                                P.spine_grp_begin.size() != P.spine_pass_begin.size()))
    return "staged spine tables do not match the passes";
  const int32_t epc = 16 / P.acc_size;
  for (size_t p = 0; p + 1 < P.spine_pass_begin.size(); p++) {
    if (P.spine_pass_smem[p] <= 0) continue;
    const int64_t b = P.spine_pass_begin[p], e = P.spine_pass_begin[p + 1];
    const int64_t ng = (e - b + kSpineRows - 1) / kSpineRows;
    if (P.spine_grp_begin[p + 1] - P.spine_grp_begin[p] != ng) return "staged spine: group count";
    for (int64_t g = 0; g < ng; g++) {
      const SpineGrp& G = P.spine_grps[P.spine_grp_begin[p] + g];
      if (G.seg_count < 1 || G.seg_count > kStageMaxSegs || G.seg_begin < 0 ||
          (size_t)G.seg_begin + G.seg_count > P.spine_segs.size())
        return "staged spine: segments of group " + std::to_string(g);
      for (int32_t s = 0; s < G.seg_count; s++) {
        const SpineSeg& S = P.spine_segs[G.seg_begin + s];
        if (S.smem % epc || S.len % epc || S.a_off % epc || S.row % epc || S.smem < 0 || S.len < kStageTile ||
            (int64_t)S.smem + S.len > P.spine_pass_smem[p])
          return "staged spine: window layout";
        if (S.row < 0 || S.wpart < 1 || S.row + S.wpart > ws_elems) return "staged spine: window row";
      }
      const int64_t r1 = std::min<int64_t>(e, b + (g + 1) * kSpineRows);
      for (int64_t r = b + g * kSpineRows; r < r1; r++) {
        const SpineRow& R = P.spine_rows[r];
        const QuadDesc& Q = P.quad[R.q];
        for (int32_t c = 0; c < R.term_count; c++) {
          const SpineTerm& T = P.spine_terms[R.term_begin + c];
          bool found = false;
          for (int32_t s = 0; s < G.seg_count && !found; s++) {
            const SpineSeg& S = P.spine_segs[G.seg_begin + s];
            found = S.row == T.row && S.wpart == T.wpart && T.sofs - S.smem == T.off - S.a_off &&
                    T.sofs >= S.smem && T.sofs + kStageTile <= S.smem + S.len;
          }
          if (!found) return at("staged spine", r) + "term outside its window";
          if (!Q.ext && Q.W < kStageTile + 4 * kStageMaxSpan) return at("staged spine", r) + "cyclic row too short";
        }
      }
    }
  }

  // ---- adjoint ----
  if (!P.has_adjoint) return "";
  const int64_t adj_elems = (int64_t)((P.adj_ws_bytes - kWsHeader) / P.acc_size);
  for (int q = 0; q < 4; q++) {
    if (!(P.cfg.quads & (1u << q))) continue;
    // view gradients sit after the forward buffers, 16-byte aligned rows
    const QuadDesc& Q = P.quad[q];
    const int64_t img = (int64_t)Q.n * grad_pitch(Q.L);
    if (Q.grad_off < ws_elems) return "adjoint gradient image overlaps the forward buffers";
    if (Q.grad_off + img > adj_elems) return "adjoint gradient image outside the workspace";
    if (Q.grad_off % 4 != 0) return "adjoint gradient image not 4-element aligned";
    if ((int64_t)Q.n * Q.L != (int64_t)P.cfg.h * P.cfg.w) return "adjoint gradient view is not the image's size";
    for (int r = 0; r < q; r++) {
      if (!(P.cfg.quads & (1u << r))) continue;
      const int64_t o = P.quad[r].grad_off, e = o + (int64_t)P.quad[r].n * grad_pitch(P.quad[r].L);
      if (Q.grad_off < e && o < Q.grad_off + img) return "adjoint gradient images overlap";
    }
  }
  for (size_t k = 0; k < P.fused.size(); k++) {
    const FusedItem& it = P.fused[k];
    const QuadDesc& Q = P.quad[it.q];
    const int32_t ATW = P.adj_tw;
    if (it.antiles < 1 || (int64_t)(it.antiles - 1) * ATW >= Q.L || (int64_t)it.antiles * ATW < Q.L)
      return at("adjoint fused", k) + "tiles do not cover the view length";
    if (it.antiles > P.max_antiles) return at("adjoint fused", k) + "more tiles than the grid";
    const int32_t TZin = ATW + it.m - 1;
    if (adj_padl + TZin > adj_rp) return at("adjoint fused", k) + "window wider than the shared row";
    if (it.aprog < 0 || (size_t)it.aprog + (size_t)it.nlev * (it.m + 1) > P.aptr.size())
      return at("adjoint fused", k) + "program pointers";
    for (int32_t l = 0; l < it.nlev; l++)
      for (int32_t r = 0; r <= it.m; r++) {
        const int32_t v = P.aptr[(size_t)it.aprog + (size_t)l * (it.m + 1) + r];
        if (v < 0 || (size_t)v > P.aops.size()) return at("adjoint fused", k) + "program terms";
        if (r < it.m) {
          const int32_t e = P.aptr[(size_t)it.aprog + (size_t)l * (it.m + 1) + r + 1];
          for (int32_t t = v; t < e; t++) {
            const MergeOp& op = P.aops[t];
            if (op.top < 0 || op.top >= it.m || op.s < 0 || op.s > adj_padl)
              return at("adjoint fused", k) + "term outside the shared window";
          }
        }
      }
  }
  for (size_t p = 0; p + 1 < P.apass_begin.size(); p++) {
    std::set<int64_t> written;
    for (int64_t k = P.apass_begin[p]; k < P.apass_begin[p + 1]; k++) written.insert(P.arows[k].dst);
    for (int64_t k = P.apass_begin[p]; k < P.apass_begin[p + 1]; k++) {
      const AdjRow& R = P.arows[k];
      const bool fin = R.flags & ROW_FINAL, ext = R.flags & ROW_EXT;
      if (R.dst < 0 || R.dst + R.wdst > ws_elems) return at("adjoint row", k) + "store outside the workspace";
      if (R.term_begin < 0 || (size_t)R.term_begin + R.term_count > P.aterms.size())
        return at("adjoint row", k) + "terms";
      for (int32_t c = 0; c < R.term_count; c++) {
        const AdjTerm& T = P.aterms[R.term_begin + c];
        if (!ext && (T.e < 0 || T.e >= R.W || R.wdst != R.W || R.wsrc != R.W))
          return at("adjoint row", k) + "cyclic offset not reduced";
        const int64_t row = R.src + (int64_t)T.t * R.src_pitch;
        if (fin) {
          if (R.src_pitch != R.W || row < 0 || row + R.W > out_elems) return at("adjoint row", k) + "source outside the output";
        } else {
          if (row < 0 || row + R.wsrc > ws_elems) return at("adjoint row", k) + "source outside the workspace";
          if (written.count(row)) return at("adjoint row", k) + "reads a row written in the same pass";
        }
      }
    }
  }
  return "";
}

}  // namespace fht

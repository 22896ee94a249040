"""A plan's tables, executed on the host, give the oracle's transform (CPU only).

`fht_plan_table` hands out the host copies of a plan's tables.  This test runs
them with numpy, in int64, exactly as the tables describe each step:

  * fused subtrees (FusedItem + their MergeOp programs): the subtree's input
    rows are read from the quadrant's view of the image at node columns
    u = x + c (zero outside the row with the extended boundary, wrapped with
    the cyclic one), then every level computes  dst[r][u] = src[top][u] +
    src[bot][u + s]  (Algorithm 1's merge with the shift of the child's
    pattern), and the rows are stored in the workspace, or through the
    quadrant's column map X = (sigma u + kappa) mod W when the subtree is the
    whole tree;
  * per-height passes (RowJob): out[u] = top[u + dtop] + bot[u + dbot], with
    indices mod W (cyclic) or zero outside the child rows (extended);
  * band schedule: band items and spine rows (SpineRow + SpineTerm):
    H[t][u] = sum_p part_p[row][u + off].

and compares the result with the oracle, element for element.  It pins the
planner's merge tables (the rounding of t -> (t1, t2, s)), its column
conventions, buffer offsets and quadrant maps without a GPU.  Band items are
checked through their own block semantics (see _run_band).
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2411_07351_gb300", "csrc")

QUAD = np.dtype({"names": ["transpose", "flip", "n", "L", "W", "ext", "sigma", "kappa", "out_off", "grad_off"],
                 "formats": ["<i4"] * 8 + ["<i8"] * 2}, align=True)
FUSED = np.dtype({"names": ["q", "a", "m", "nlev", "prog", "wn", "c", "final_", "dst", "dst_pitch", "ntiles",
                            "aprog", "antiles", "kind", "tw", "L", "B", "K0", "wsrc", "c_src", "src_pitch", "src"],
                  "formats": ["<i4"] * 8 + ["<i8"] + ["<i4"] * 12 + ["<i8"]}, align=True)
MERGE = np.dtype({"names": ["top", "bot", "s", "pad"], "formats": ["<i2"] * 4}, align=True)
ROW = np.dtype({"names": ["dst", "top", "bot", "wout", "wtop", "wbot", "dtop", "dbot", "W", "flags", "kappa"],
                "formats": ["<i8"] * 3 + ["<i4"] * 8}, align=True)
SPINE_ROW = np.dtype({"names": ["dst", "q", "term_begin", "term_count", "flags", "w", "pad"],
                      "formats": ["<i8"] + ["<i4"] * 6}, align=True)
SPINE_TERM = np.dtype({"names": ["row", "wpart", "off", "sofs", "pad"], "formats": ["<i8"] + ["<i4"] * 4},
                      align=True)
DTYPES = {"QuadDesc": QUAD, "FusedItem": FUSED, "MergeOp": MERGE, "RowJob": ROW, "SpineRow": SPINE_ROW,
          "SpineTerm": SPINE_TERM}

ROW_FINAL, ROW_EXT, ROW_NEG = 1, 2, 4
SPINE_INNER = 1
FUSED_GENERIC, FUSED_BY64, FUSED_BAND = 0, 1, 2


@pytest.fixture(scope="module")
def F():
    from paper_2411_07351_gb300 import build as B

    B.build()
    import paper_2411_07351_gb300 as F

    return F


def test_descriptor_layouts_match_the_header(tmp_path):
    gxx = shutil.which("g++") or shutil.which("c++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    lines = ["#include <cstdio>", "#include <cstddef>", '#include "fht_desc.h"', "int main() {"]
    for name, dt in DTYPES.items():
        lines.append(f'  std::printf("size {name} %zu\\n", sizeof(fht::{name}));')
        for f in dt.names:
            lines.append(f'  std::printf("off {name}.{f} %zu\\n", offsetof(fht::{name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "probe.cpp"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run([gxx, "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True, capture_output=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        kind, key, val = ln.split()
        got[(kind, key)] = int(val)
    for name, dt in DTYPES.items():
        assert dt.itemsize == got[("size", name)], name
        for f in dt.names:
            assert dt.fields[f][1] == got[("off", f"{name}.{f}")], f"{name}.{f}"


def _table(F, plan, which, dtype):
    from paper_2411_07351_gb300 import _capi as C

    data, count, esz = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_int32()
    C.check(C.load().fht_plan_table(plan._h, which, ctypes.byref(data), ctypes.byref(count), ctypes.byref(esz)),
            "fht_plan_table")
    assert esz.value == dtype.itemsize
    if count.value == 0:
        return np.zeros(0, dtype=dtype)
    buf = (ctypes.c_char * (count.value * esz.value)).from_address(data.value)
    return np.frombuffer(bytes(buf), dtype=dtype)


def _tables(F, plan):
    from paper_2411_07351_gb300 import _capi as C

    return {
        "quads": _table(F, plan, C.FHT_TABLE_QUADS, QUAD),
        "fused": _table(F, plan, C.FHT_TABLE_FUSED, FUSED),
        "ops": _table(F, plan, C.FHT_TABLE_OPS, MERGE),
        "rows": _table(F, plan, C.FHT_TABLE_ROWS, ROW),
        "pass_begin": _table(F, plan, C.FHT_TABLE_PASS_BEGIN, np.dtype("<i8")),
        "band_items": _table(F, plan, C.FHT_TABLE_BAND_ITEMS, FUSED),
        "spine_rows": _table(F, plan, C.FHT_TABLE_SPINE_ROWS, SPINE_ROW),
        "spine_terms": _table(F, plan, C.FHT_TABLE_SPINE_TERMS, SPINE_TERM),
        "spine_begin": _table(F, plan, C.FHT_TABLE_SPINE_BEGIN, np.dtype("<i8")),
    }


def _view(img, Q):
    V = img.T if Q["transpose"] else img
    return V[:, ::-1] if Q["flip"] else V


def _read_view(V, rows, x, ext):
    """V[rows][x] for any integer columns x: zero outside [0, L) (extended) or wrapped (cyclic)."""
    L = V.shape[1]
    if ext:
        ok = (x >= 0) & (x < L)
        vals = V[np.ix_(rows, np.clip(x, 0, L - 1))]
        return np.where(ok[None, :], vals, 0)
    return V[np.ix_(rows, np.mod(x, L))]


def _shifted(v, s):
    """v[j + s] for j in [0, len(v)), zero past the end (columns the stored rows never reach)."""
    if s == 0:
        return v
    out = np.zeros_like(v)
    out[: len(v) - s] = v[s:]
    return out


def _store(out, ws, Q, final, dst, pitch, r, vals, u):
    if final:
        X = np.mod(Q["sigma"] * u + Q["kappa"], Q["W"])
        out[dst + r * pitch + X] = vals
    else:
        ws[dst + r * pitch + u] = vals


def _run_fused(T, img, out, ws):
    for it in T["fused"]:
        Q = T["quads"][it["q"]]
        V = _view(img, Q)
        m, c, wn = int(it["m"]), int(it["c"]), int(it["wn"])
        u = np.arange(wn + m)
        cur = _read_view(V, np.arange(it["a"], it["a"] + m), u - c, Q["ext"]).astype(np.int64)
        prog = T["ops"][it["prog"]: it["prog"] + it["nlev"] * m].reshape(it["nlev"], m) if it["nlev"] else []
        for lev in prog:
            nxt = np.empty_like(cur)
            for r, op in enumerate(lev):
                nxt[r] = cur[op["top"]] if op["bot"] < 0 else cur[op["top"]] + _shifted(cur[op["bot"]], op["s"])
            cur = nxt
        for r in range(m):
            _store(out, ws, Q, it["final_"], int(it["dst"]), int(it["dst_pitch"]), r, cur[r, :wn], u[:wn])


def _run_rows(T, out, ws):
    pb = T["pass_begin"]
    for p in range(len(pb) - 1):
        for J in T["rows"][pb[p]: pb[p + 1]]:
            u = np.arange(J["wout"])
            if J["flags"] & ROW_EXT:
                i1, i2 = u + J["dtop"], u + J["dbot"]
                a = np.where((i1 >= 0) & (i1 < J["wtop"]), ws[J["top"] + np.clip(i1, 0, J["wtop"] - 1)], 0)
                b = np.where((i2 >= 0) & (i2 < J["wbot"]), ws[J["bot"] + np.clip(i2, 0, J["wbot"] - 1)], 0)
            else:
                a = ws[J["top"] + np.mod(u + J["dtop"], J["W"])]
                b = ws[J["bot"] + np.mod(u + J["dbot"], J["W"])]
            v = a + b
            if J["flags"] & ROW_FINAL:
                X = J["kappa"] - u if J["flags"] & ROW_NEG else u + J["kappa"]
                out[J["dst"] + np.mod(X, J["W"])] = v
            else:
                ws[J["dst"] + u] = v


def _execute(F, plan, img):
    T = _tables(F, plan)
    out = np.full(plan.out_elems, -(1 << 60), dtype=np.int64)  # every element must be written
    ws = np.zeros((plan.workspace_bytes - 256) // 4, dtype=np.int64)
    _run_fused(T, img.astype(np.int64), out, ws)
    if len(T["spine_rows"]) or len(T["band_items"]):
        _run_band(T, out, ws)
        _run_spine(T, out, ws)
    else:
        _run_rows(T, out, ws)
    return out


PER_HEIGHT = [(h, w, b, s, fr) for (h, w) in [(1, 1), (1, 7), (9, 1), (3, 5), (17, 13), (45, 70), (100, 37),
                                               (130, 66), (257, 31)]
              for b in ("cyclic", "extended") for (s, fr) in (("S", 0), ("T", 16), ("T", 32), ("S", 8))]


@pytest.mark.parametrize("h,w,boundary,split,fused_rows", PER_HEIGHT)
def test_per_height_tables_give_the_oracle_transform(F, orc, h, w, boundary, split, fused_rows):
    import torch

    rng = np.random.default_rng(h * 1000 + w)
    img = rng.integers(0, 256, size=(h, w)).astype(np.uint8)
    plan = F.Plan(h, w, torch.uint8, F.FHT_QALL, boundary, split=split, fused_rows=fused_rows, device=-1)
    T = _tables(F, plan)
    assert len(T["spine_rows"]) == 0 and len(T["band_items"]) == 0
    got = _execute(F, plan, img)
    ref = orc.fht(img.astype(np.int64), 15, orc.EXTENDED if boundary == "extended" else orc.CYCLIC,
                  orc.SPLIT_S if split == "S" else orc.SPLIT_T)
    assert np.array_equal(got, ref), f"{(got != ref).sum()} of {got.size} differ"


def _read_row(ws, base, width, z, ext):
    """Row values at columns z of a width-column workspace row: zero outside it
    (extended) or wrapped (cyclic)."""
    if ext:
        ok = (z >= 0) & (z < width)
        return np.where(ok, ws[base + np.clip(z, 0, width - 1)], 0)
    return ws[base + np.mod(z, width)]


def _run_band(T, out, ws):
    # A band item: a perfect band of B = 2^L blocks of 64 rows.  Its group g
    # (block row K = K0 + g) stages row K of every block b at block column
    # x + c_src + K b, merges the B staged rows as a B-row Brady-Yong block
    # (t = 2k + i: rows k of both halves, shift k + i), and stores output rows
    # K B + i of the band at node columns u = x + c.
    for it in T["band_items"]:
        Q = T["quads"][it["q"]]
        B, c, wn = int(it["B"]), int(it["c"]), int(it["wn"])
        G = 64 // B
        u = np.arange(wn + B)
        x = u - c
        for g in range(G):
            K = int(it["K0"]) + g
            rows = [_read_row(ws, int(it["src"]) + (64 * b + K) * int(it["src_pitch"]), int(it["wsrc"]),
                              x + int(it["c_src"]) + K * b, Q["ext"]) for b in range(B)]
            M = 1
            while M < B:
                nxt = []
                for j0 in range(0, B, 2 * M):
                    lo, hi = rows[j0: j0 + M], rows[j0 + M: j0 + 2 * M]
                    for t in range(2 * M):
                        k, i = t // 2, t % 2
                        nxt.append(lo[k] + _shifted(hi[k], k + i))
                rows = nxt
                M *= 2
            for i in range(B):
                _store(out, ws, Q, it["final_"], int(it["dst"]), int(it["dst_pitch"]), g * B + i, rows[i][:wn],
                       u[:wn])


def _run_spine(T, out, ws):
    sb, terms = T["spine_begin"], T["spine_terms"]
    for p in range(len(sb) - 1):
        for R in T["spine_rows"][sb[p]: sb[p + 1]]:
            Q = T["quads"][R["q"]]
            u = np.arange(R["w"])
            acc = np.zeros(R["w"], dtype=np.int64)
            for S in terms[R["term_begin"]: R["term_begin"] + R["term_count"]]:
                acc += _read_row(ws, int(S["row"]), int(S["wpart"]), u + int(S["off"]), Q["ext"])
            if R["flags"] & SPINE_INNER:
                ws[R["dst"] + u] = acc
            else:
                out[R["dst"] + np.mod(Q["sigma"] * u + Q["kappa"], Q["W"])] = acc


BAND = [(h, w, b) for (h, w) in [(65, 9), (128, 40), (131, 45), (200, 150), (300, 77), (513, 20), (700, 260)]
        for b in ("cyclic", "extended")]


@pytest.mark.parametrize("h,w,boundary", BAND)
def test_band_schedule_tables_give_the_oracle_transform(F, orc, h, w, boundary):
    import torch

    rng = np.random.default_rng(h * 1000 + w + 7)
    img = rng.integers(0, 256, size=(h, w)).astype(np.uint8)
    plan = F.Plan(h, w, torch.uint8, F.FHT_QALL, boundary, device=-1)
    T = _tables(F, plan)
    assert len(T["spine_rows"]) > 0 or len(T["band_items"]) > 0
    got = _execute(F, plan, img)
    ref = orc.fht(img.astype(np.int64), 15, orc.EXTENDED if boundary == "extended" else orc.CYCLIC)
    assert np.array_equal(got, ref), f"{(got != ref).sum()} of {got.size} differ"


@pytest.mark.parametrize("chunk", [1, 2, 4])
@pytest.mark.parametrize("boundary", ["cyclic", "extended"])
def test_spine_chunks_tables_give_the_oracle_transform(F, orc, chunk, boundary):
    import torch

    h, w = 1500, 30  # spine 1024 + 256 + 128 + 64 + 28: inner chunk tops for every chunk size here
    img = np.random.default_rng(11).integers(0, 256, size=(h, w)).astype(np.uint8)
    plan = F.Plan(h, w, torch.uint8, F.FHT_Q0 | F.FHT_Q1, boundary, spine_chunk=chunk, device=-1)
    got = _execute(F, plan, img)
    ref = orc.fht(img.astype(np.int64), 3, orc.EXTENDED if boundary == "extended" else orc.CYCLIC)
    assert np.array_equal(got, ref)


def test_root_taller_than_8192_rows(F, orc):
    import torch

    # Q0/Q1 split 8300 rows: the 8192-row part is "big" (summed first from its
    # 4096-row bands); cyclic keeps the rows 3 columns wide
    h, w = 8300, 3
    img = np.random.default_rng(12).integers(0, 256, size=(h, w)).astype(np.uint8)
    plan = F.Plan(h, w, torch.uint8, F.FHT_Q0 | F.FHT_Q1, "cyclic", device=-1)
    got = _execute(F, plan, img)
    ref = orc.fht(img.astype(np.int64), 3, orc.CYCLIC)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("h,w,differ", [(23, 30, True), (91, 20, True), (45, 17, False), (181, 64, False)])
def test_tables_follow_the_rounding_rule(F, orc, h, w, differ):
    """The same plan shape under the two readings of the child slopes (exact
    ties to even, and k_P in double): each plan's tables match the oracle under
    its own rule.  At 23 x 30 and 91 x 20 the two transforms differ (a tie
    decides a child slope), so the comparison does see the merge tables; at
    the other two every tie's double product rounds (half to even) the way
    the exact rule does."""
    import torch

    img = np.random.default_rng(h + w).integers(0, 256, size=(h, w)).astype(np.uint8)
    exact = _execute(F, F.Plan(h, w, torch.uint8, 15, "extended", device=-1), img)
    orc.set_rounding(orc.ROUND_FLOAT)
    try:
        ref_float = orc.fht(img.astype(np.int64), 15, orc.EXTENDED)
    finally:
        orc.set_rounding(orc.ROUND_EXACT)
    flt = _execute(F, F.Plan(h, w, torch.uint8, 15, "extended", rounding="float", device=-1), img)
    assert np.array_equal(exact, orc.fht(img.astype(np.int64), 15, orc.EXTENDED))
    assert np.array_equal(flt, ref_float)
    assert np.array_equal(exact, flt) != differ


ADJ_ROW = np.dtype({"names": ["dst", "src", "src_pitch", "wdst", "wsrc", "W", "flags", "kappa", "term_begin",
                              "term_count"], "formats": ["<i8"] * 2 + ["<i4"] * 8}, align=True)
ADJ_TERM = np.dtype({"names": ["t", "e"], "formats": ["<i4"] * 2}, align=True)
DTYPES.update({"AdjRow": ADJ_ROW, "AdjTerm": ADJ_TERM})


def _adjoint_tables(F, plan):
    from paper_2411_07351_gb300 import _capi as C

    T = _tables(F, plan)
    T.update({
        "arows": _table(F, plan, C.FHT_TABLE_ADJ_ROWS, ADJ_ROW),
        "aterms": _table(F, plan, C.FHT_TABLE_ADJ_TERMS, ADJ_TERM),
        "abegin": _table(F, plan, C.FHT_TABLE_ADJ_BEGIN, np.dtype("<i8")),
        "aptr": _table(F, plan, C.FHT_TABLE_ADJ_PTR, np.dtype("<i4")),
        "aops": _table(F, plan, C.FHT_TABLE_ADJ_OPS, MERGE),
    })
    return T


def _execute_adjoint(F, plan, gout):
    """The adjoint schedule from the tables: per-height gather passes (highest
    first), then every fused subtree's levels in reverse into the quadrants'
    view gradients, then their sum mapped back onto the image."""
    T = _adjoint_tables(F, plan)
    h, w = plan.h, plan.w
    ws = np.zeros((plan.adjoint_workspace_bytes - 256) // 4, dtype=np.int64)
    ab, terms = T["abegin"], T["aterms"]
    for p in range(len(ab) - 1):
        for R in T["arows"][ab[p]: ab[p + 1]]:
            src = gout if R["flags"] & ROW_FINAL else ws
            i = np.arange(R["wdst"])
            acc = np.zeros(R["wdst"], dtype=np.int64)
            for k in terms[R["term_begin"]: R["term_begin"] + R["term_count"]]:
                u = i + k["e"]
                if R["flags"] & ROW_EXT:
                    ok = (u >= 0) & (u < R["wsrc"])
                else:
                    ok = np.ones_like(u, dtype=bool)
                    u = np.mod(u, R["W"])
                if R["flags"] & ROW_FINAL:
                    u = np.mod(R["kappa"] - u if R["flags"] & ROW_NEG else u + R["kappa"], R["W"])
                vals = src[R["src"] + k["t"] * int(R["src_pitch"]) + np.clip(u, 0, None)]
                acc += np.where(ok, vals, 0)
            ws[R["dst"] + i] = acc
    for it in T["fused"]:
        Q = T["quads"][it["q"]]
        m, c, wn, L = int(it["m"]), int(it["c"]), int(it["wn"]), int(Q["L"])
        x = np.arange(-(m - 1), L)  # view columns: the gradient reaches m - 1 columns left of the row
        u = x + c
        ok = (u >= 0) & (u < wn) if Q["ext"] else np.ones_like(u, dtype=bool)
        u = np.clip(u, 0, wn - 1) if Q["ext"] else np.mod(u, Q["W"])
        cur = np.zeros((m, len(x)), dtype=np.int64)
        for r in range(m):
            if it["final_"]:
                X = np.mod(Q["sigma"] * u + Q["kappa"], Q["W"])
                cur[r] = np.where(ok, gout[it["dst"] + r * Q["W"] + X], 0)
            else:
                cur[r] = np.where(ok, ws[it["dst"] + r * it["dst_pitch"] + u], 0)
        for lev in range(it["nlev"] - 1, -1, -1):
            ptr = T["aptr"][it["aprog"] + lev * (m + 1): it["aprog"] + (lev + 1) * (m + 1)]
            nxt = np.zeros_like(cur)
            for k in range(m):
                for op in T["aops"][ptr[k]: ptr[k + 1]]:
                    s = int(op["s"])
                    nxt[k, s:] += cur[op["top"], : len(x) - s]  # g[k][j] += g'[top][j - s]
            cur = nxt
        z = np.arange(L)
        gp = (L + 3) // 4 * 4  # view gradient rows: L elements padded to a multiple of 4
        for r in range(m):
            ws[Q["grad_off"] + (it["a"] + r) * gp + z] = cur[r, z + m - 1]
    gin = np.zeros((h, w), dtype=np.int64)
    for q in range(4):
        if plan.quads & (1 << q):
            Q = T["quads"][q]
            off, n, L = int(Q["grad_off"]), int(Q["n"]), int(Q["L"])
            gp = (L + 3) // 4 * 4
            assert off % 4 == 0
            g = ws[off: off + n * gp].reshape(n, gp)[:, :L]  # view gradient gV[r][z]
            if Q["flip"]:
                g = g[:, ::-1]
            gin += g.T if Q["transpose"] else g
    return gin


ADJ = [(h, w, b, s, fr) for (h, w) in [(1, 1), (1, 6), (7, 1), (5, 3), (17, 13), (40, 70), (100, 37), (131, 45)]
       for b in ("cyclic", "extended") for (s, fr) in (("T", 0), ("S", 0), ("T", 16))]


@pytest.mark.parametrize("h,w,boundary,split,fused_rows", ADJ)
def test_adjoint_tables_give_the_oracle_adjoint(F, orc, h, w, boundary, split, fused_rows):
    import torch

    plan = F.Plan(h, w, torch.uint8, F.FHT_QALL, boundary, split=split, fused_rows=fused_rows, with_adjoint=True,
                  device=-1)
    gout = np.random.default_rng(h * 31 + w).integers(-50, 50, size=plan.out_elems).astype(np.int64)
    got = _execute_adjoint(F, plan, gout)
    ref = orc.adjoint(gout.astype(np.float64), h, w, 15, orc.EXTENDED if boundary == "extended" else orc.CYCLIC,
                      orc.SPLIT_S if split == "S" else orc.SPLIT_T)
    assert np.array_equal(got, ref.astype(np.int64)), f"{(got != ref).sum()} of {got.size} differ"


def _sweep(n, seed):
    rng = np.random.default_rng(seed)
    cases = []
    for _ in range(n):
        h, w = (int(v) for v in rng.integers(1, 400, size=2))
        split = "S" if rng.random() < 0.3 else "T"
        fr = int(rng.choice([0, 0, 8, 16, 32]))
        boundary = "extended" if rng.random() < 0.5 else "cyclic"
        quads = int(rng.integers(1, 16))
        cases.append((h, w, boundary, split, fr, quads))
    return cases


@pytest.mark.parametrize("h,w,boundary,split,fused_rows,quads", _sweep(30, 2024))
def test_random_shapes_forward_and_adjoint(F, orc, h, w, boundary, split, fused_rows, quads):
    import torch

    b = orc.EXTENDED if boundary == "extended" else orc.CYCLIC
    rule = orc.SPLIT_S if split == "S" else orc.SPLIT_T
    plan = F.Plan(h, w, torch.uint8, quads, boundary, split=split, fused_rows=fused_rows, with_adjoint=True,
                  device=-1)
    rng = np.random.default_rng(h * 7919 + w)
    img = rng.integers(0, 256, size=(h, w)).astype(np.uint8)
    assert np.array_equal(_execute(F, plan, img), orc.fht(img.astype(np.int64), quads, b, rule))
    gout = rng.integers(-50, 50, size=plan.out_elems).astype(np.int64)
    ref = orc.adjoint(gout.astype(np.float64), h, w, quads, b, rule)
    assert np.array_equal(_execute_adjoint(F, plan, gout), ref.astype(np.int64))


@pytest.mark.parametrize("split", ["T", "S"])
@pytest.mark.parametrize("boundary", ["cyclic", "extended"])
def test_64_row_blocks_are_classical_brady_yong(F, split, boundary):
    """The 64-row block kernel does not read its program: it merges adjacent
    blocks of M rows as  out[2M g + t] = in[2M g + t//2] + in[2M g + M + t//2]
    shifted by ceil(t/2), six times.  Every 64-row item's program in the plan
    (which the host interpreter above runs and checks against the oracle) must
    be exactly that."""
    import torch

    # Split_S halves, so it makes 64-row subtrees only under heights 64 * 2^k
    h, w = (300, 200) if split == "T" else (256, 320)
    plan = F.Plan(h, w, torch.uint8, 15, boundary, split=split, device=-1)
    T = _tables(F, plan)
    items = [it for it in T["fused"] if it["kind"] == FUSED_BY64]
    assert items and all(it["m"] == 64 and it["nlev"] == 6 for it in items)
    for it in items:
        prog = T["ops"][it["prog"]: it["prog"] + 6 * 64].reshape(6, 64)
        for lev in range(6):
            M = 1 << lev
            for r in range(64):
                g, t = divmod(r, 2 * M)
                op = prog[lev][r]
                assert (op["top"], op["bot"], op["s"]) == (2 * M * g + t // 2, 2 * M * g + M + t // 2, (t + 1) // 2)


def _launch_bytes_from_tables(T, in_size, acc, vblock=False):
    """Compulsory bytes of every forward launch, counted from the tables: the
    distinct rows a launch reads (each at its row width) and the rows it
    writes, once each.  With the register-tiled block path the generic
    subtrees (if any) and the 64-row blocks are two launches."""
    Qs = T["quads"]

    def item_bytes(it):
        return int(it["m"]) * int(Qs[it["q"]]["L"]) * in_size + int(it["m"]) * int(it["wn"]) * acc

    if vblock:
        gen = [item_bytes(it) for it in T["fused"] if int(it["kind"]) == 0]
        launches = ([sum(gen)] if gen else []) + [sum(item_bytes(it) for it in T["fused"] if int(it["kind"]) != 0)]
    else:
        launches = [sum(item_bytes(it) for it in T["fused"])]
    if len(T["band_items"]) or len(T["spine_rows"]):
        if len(T["band_items"]):
            reads, writes = set(), 0
            for it in T["band_items"]:
                B, G = int(it["B"]), 64 // int(it["B"])
                for g in range(G):
                    for b in range(B):
                        reads.add((int(it["src"]) + (64 * b + int(it["K0"]) + g) * int(it["src_pitch"]),
                                   int(it["wsrc"])))
                writes += G * B * int(it["wn"])
            launches.append((sum(wd for _, wd in reads) + writes) * acc)
        sb, terms = T["spine_begin"], T["spine_terms"]
        for p in range(len(sb) - 1):
            rows = T["spine_rows"][sb[p]: sb[p + 1]]
            if len(rows) == 0:
                continue
            reads = {(int(S["row"]), int(S["wpart"])) for R in rows
                     for S in terms[R["term_begin"]: R["term_begin"] + R["term_count"]]}
            launches.append((sum(wd for _, wd in reads) + sum(int(R["w"]) for R in rows)) * acc)
    else:
        pb = T["pass_begin"]
        for p in range(len(pb) - 1):
            rows = T["rows"][pb[p]: pb[p + 1]]
            if len(rows) == 0:
                continue
            reads = {(int(J["top"]), int(J["wtop"])) for J in rows} | {(int(J["bot"]), int(J["wbot"])) for J in rows}
            launches.append((sum(wd for _, wd in reads) + sum(int(J["wout"]) for J in rows)) * acc)
    return launches


@pytest.mark.parametrize("h,w,boundary,split,dtype", [
    (4095, 4095, "extended", "T", "float32"), (4095, 4095, "cyclic", "T", "float32"),
    (2047, 300, "extended", "T", "uint8"), (8300, 3, "cyclic", "T", "uint8"),
    (1000, 700, "extended", "S", "float32"), (257, 257, "cyclic", "T", "uint8"), (4096, 640, "cyclic", "T", "uint8")])
@pytest.mark.parametrize("tile", [(128, 512), (192, 256)])
def test_launch_model_bytes_match_the_tables(F, h, w, boundary, split, dtype, tile):
    """The per-launch model bytes the bench divides by each launch's time
    (fht_plan_launch_info) equal the distinct rows each launch reads and
    writes according to its own tables."""
    import torch

    from paper_2411_07351_gb300 import _capi as C

    tdt = {"float32": torch.float32, "uint8": torch.uint8}[dtype]
    plan = F.Plan(h, w, tdt, F.FHT_QALL, boundary, split=split, device=-1, tile_cols=tile[0], threads=tile[1])
    T = _tables(F, plan)
    vblock = tile == (192, 256) and any(int(it["kind"]) == 1 for it in T["fused"])
    want = _launch_bytes_from_tables(T, 4 if dtype == "float32" else 1, 4, vblock)
    lib = C.load()
    n = ctypes.c_int32()
    C.check(lib.fht_plan_launches(plan._h, ctypes.byref(n)), "fht_plan_launches")
    got = []
    for k in range(n.value):
        kind, by = ctypes.c_int32(), ctypes.c_int64()
        C.check(lib.fht_plan_launch_info(plan._h, k, ctypes.byref(kind), ctypes.byref(by)), "fht_plan_launch_info")
        got.append(by.value)
    assert got == want
    assert sum(got) == plan.info.model_bytes


@pytest.mark.parametrize("n", [2, 3, 5, 17, 64, 100, 257, 1000])
@pytest.mark.parametrize("split,fused_rows", [("T", 32), ("T", 8), ("S", 0)])
def test_executed_additions_are_theorem_1(F, orc, n, split, fused_rows):
    """Cyclic, one quadrant, per-height schedule: every merged row is one
    addition per column, so the additions the tables perform (fused programs'
    merged rows and per-height rows, W columns each) are Theorem 1's f(n)."""
    import torch

    plan = F.Plan(n, n, torch.uint8, F.FHT_Q0, "cyclic", split=split, fused_rows=fused_rows, device=-1)
    T = _tables(F, plan)
    assert len(T["spine_rows"]) == 0
    W = n
    merged = 0
    for it in T["fused"]:
        ops = T["ops"][it["prog"]: it["prog"] + it["nlev"] * it["m"]]
        merged += int((ops["bot"] >= 0).sum())
    merged += len(T["rows"])
    rule = orc.SPLIT_S if split == "S" else orc.SPLIT_T
    assert merged * W == orc.adds(n, rule) == plan.info.adds

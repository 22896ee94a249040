/*
 * Plain, slow CPU oracle for the generalised Brady-Yong fast Hough transform
 * (FHT2DT, and the FHT2DS variant it is compared with).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or table with the CUDA path.
 *
 * Paper: "Generalization of Brady-Yong Algorithm for Fast Hough Transform to
 * Arbitrary Image Size" (arXiv 2411.07351).
 *
 * Orientation.  The paper splits the image width and rotates along the
 * height.  Here the image is row-major I[y][x] with h rows and the split runs
 * over the rows, so each Hough row J[t][:] is a contiguous vector along x and
 * Rotate acts on it.  This is the paper's Algorithm 1 applied to the
 * transposed image, written in the transposed coordinates.
 *
 * Readings of the paper taken here (each is pinned by a test):
 *  - [.] rounds half to even, computed exactly in integers (Algorithm 1 and
 *    Algorithm 2 leave the tie rule open; this rule reproduces the 36.38 %
 *    figure of Section 5).
 *  - Rotate(v, r)[i] = v[(i + r) mod len]: forced by Algorithm 2, where the
 *    right part of a pattern is displaced by +(t - t_P(1)).
 *  - Quadrants (not in the paper): Q0 shifts by +p, Q1 by -p, Q2/Q3 are Q0/Q1
 *    of the transposed image.
 *  - EXTENDED boundary (not in the paper): the cyclic transform of the image
 *    zero-padded on the right to width w + h - 1.
 *
 * All arithmetic is int64 (integer images) or double (float images).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_SPLIT_T 0
#define ORC_SPLIT_S 1
#define ORC_CYCLIC 0
#define ORC_EXTENDED 1

/* ---------------------------------------------------------------------- */
/* Section 3: the two split rules.                                        */
/*   Split_S(n) = < floor(n/2), ceil(n/2) >                               */
/*   Split_T(n) = < 2^(ceil(log2 n) - 1), n - 2^(ceil(log2 n) - 1) >      */
/* ---------------------------------------------------------------------- */
static int ceil_log2_i64(int64_t n) {
  int k = 0;
  while (((int64_t)1 << k) < n) k++;
  return k;
}

void orc_split(int32_t n, int32_t split, int32_t out[2]) {
  if (split == ORC_SPLIT_T) {
    int64_t p = (int64_t)1 << (ceil_log2_i64(n) - 1);
    out[0] = (int32_t)p;
    out[1] = (int32_t)(n - p);
  } else {
    out[0] = n / 2;
    out[1] = n - n / 2;
  }
}

/* [a / d] for a >= 0, d > 0: nearest integer, ties to even. */
int64_t orc_round_half_even(int64_t a, int64_t d) {
  int64_t q = a / d, r = a % d;
  if (2 * r > d) return q + 1;
  if (2 * r < d) return q;
  return q + (q & 1);
}

/* Rounding of the child slopes.  0 (default): [x] = nearest integer to the
 * exact rational, ties to even.  1: Algorithm 1 read literally in floating
 * point -- k_P = (n_P - 1)/(n - 1) as a double, then t k_P rounded to the
 * nearest integer (ties to even, the default FP mode) with rint. */
static int g_rounding = 0;
void orc_set_rounding(int32_t rule) { g_rounding = rule; }

/* The child slopes of Algorithm 1 / Algorithm 2: t_P = [t (n_P - 1) / (n - 1)]. */
static void child_slopes(int32_t n, const int32_t np[2], int32_t t, int32_t tp[2]) {
  if (g_rounding == 1) {
    for (int i = 0; i < 2; i++) {
      double k = (double)(np[i] - 1) / (double)(n - 1);
      tp[i] = (int32_t)rint((double)t * k);
    }
    return;
  }
  tp[0] = (int32_t)orc_round_half_even((int64_t)t * (np[0] - 1), n - 1);
  tp[1] = (int32_t)orc_round_half_even((int64_t)t * (np[1] - 1), n - 1);
}

static int32_t imod(int64_t a, int64_t m) {
  int64_t r = a % m;
  return (int32_t)(r < 0 ? r + m : r);
}

/* One child slope under the current rounding rule (for tests). */
int32_t orc_child_slope(int32_t n, int32_t ni, int32_t t) {
  int32_t np[2] = {ni, ni}, tp[2];
  child_slopes(n, np, t, tp);
  return tp[0];
}

/* ---------------------------------------------------------------------- */
/* Algorithm 2 (FHT2D_Pattern): the generating pattern pat(n, t).         */
/* pat = pat(n0, t0) ++ (pat(n1, t1) + (t - t1)).                          */
/* ---------------------------------------------------------------------- */
void orc_pattern(int32_t n, int32_t t, int32_t split, int32_t* pat) {
  if (n == 1) {
    pat[0] = 0;
    return;
  }
  int32_t np[2], tp[2];
  orc_split(n, split, np);
  child_slopes(n, np, t, tp);
  orc_pattern(np[0], tp[0], split, pat);
  orc_pattern(np[1], tp[1], split, pat + np[0]);
  for (int32_t i = 0; i < np[1]; i++) pat[np[0] + i] += t - tp[1];
}

/* Section 4: orthotropic error of pat(n, t) against y = x t / (n - 1),
 * returned as the exact numerator max_x |x t - pat(x) (n - 1)|; the error is
 * that value divided by (n - 1).  E(n) is the maximum over t.
 * For speed the two child pattern tables of Algorithm 2 are built once (all
 * slopes of each child) and every pat(n, t) is assembled from them exactly as
 * Algorithm 2's concatenation step does. */
int64_t orc_pattern_error_num(int32_t n, int32_t split) {
  if (n <= 1) return 0;
  int32_t np[2];
  orc_split(n, split, np);
  int32_t* tab0 = (int32_t*)malloc(sizeof(int32_t) * (size_t)np[0] * np[0]);
  int32_t* tab1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)np[1] * np[1]);
  for (int32_t t = 0; t < np[0]; t++) orc_pattern(np[0], t, split, tab0 + (size_t)t * np[0]);
  for (int32_t t = 0; t < np[1]; t++) orc_pattern(np[1], t, split, tab1 + (size_t)t * np[1]);
  int64_t best = 0;
  for (int32_t t = 0; t < n; t++) {
    int32_t tp[2];
    child_slopes(n, np, t, tp);
    const int32_t* p0 = tab0 + (size_t)tp[0] * np[0];
    const int32_t* p1 = tab1 + (size_t)tp[1] * np[1];
    for (int32_t x = 0; x < n; x++) {
      int64_t py = x < np[0] ? p0[x] : (int64_t)p1[x - np[0]] + (t - tp[1]);
      int64_t d = (int64_t)x * t - py * (n - 1);
      if (d < 0) d = -d;
      if (d > best) best = d;
    }
  }
  free(tab0);
  free(tab1);
  return best;
}

/* Theorem 1 proof: a node of width m costs m * n additions; the total is n
 * times the sum of the values of the non-leaf nodes of the calculation-order
 * tree G(n).  Returned here is that sum (multiply by the row length). */
int64_t orc_tree_nonleaf_sum(int32_t n, int32_t split) {
  if (n <= 1) return 0;
  int32_t np[2];
  orc_split(n, split, np);
  return (int64_t)n + orc_tree_nonleaf_sum(np[0], split) + orc_tree_nonleaf_sum(np[1], split);
}

/* ---------------------------------------------------------------------- */
/* Algorithm 1 (FHT2D), build orientation: n rows of length W, cyclic.    */
/* sign = +1: J(t,:) = R0 + Rotate(R1, t - t1); sign = -1: the mirror      */
/* quadrant, Rotate by -(t - t1).                                          */
/* ---------------------------------------------------------------------- */
static void fht_rec_i64(int32_t n, int32_t W, const int64_t* I, int64_t* J, int32_t split, int sign) {
  if (n == 1) {
    memcpy(J, I, sizeof(int64_t) * (size_t)W);
    return;
  }
  int32_t np[2];
  orc_split(n, split, np);
  int64_t* J0 = (int64_t*)malloc(sizeof(int64_t) * (size_t)np[0] * W);
  int64_t* J1 = (int64_t*)malloc(sizeof(int64_t) * (size_t)np[1] * W);
  fht_rec_i64(np[0], W, I, J0, split, sign);
  fht_rec_i64(np[1], W, I + (size_t)np[0] * W, J1, split, sign);
  memset(J, 0, sizeof(int64_t) * (size_t)n * W); /* Create_Zeroed_Image */
  for (int32_t t = 0; t < n; t++) {
    int32_t tp[2];
    child_slopes(n, np, t, tp);
    const int64_t* r0 = J0 + (size_t)tp[0] * W;
    const int64_t* r1 = J1 + (size_t)tp[1] * W;
    int64_t rot = (int64_t)sign * (t - tp[1]);
    for (int32_t x = 0; x < W; x++) J[(size_t)t * W + x] = r0[x] + r1[imod(x + rot, W)];
  }
  free(J0);
  free(J1);
}

static void fht_rec_f64(int32_t n, int32_t W, const double* I, double* J, int32_t split, int sign) {
  if (n == 1) {
    memcpy(J, I, sizeof(double) * (size_t)W);
    return;
  }
  int32_t np[2];
  orc_split(n, split, np);
  double* J0 = (double*)malloc(sizeof(double) * (size_t)np[0] * W);
  double* J1 = (double*)malloc(sizeof(double) * (size_t)np[1] * W);
  fht_rec_f64(np[0], W, I, J0, split, sign);
  fht_rec_f64(np[1], W, I + (size_t)np[0] * W, J1, split, sign);
  memset(J, 0, sizeof(double) * (size_t)n * W);
  for (int32_t t = 0; t < n; t++) {
    int32_t tp[2];
    child_slopes(n, np, t, tp);
    const double* r0 = J0 + (size_t)tp[0] * W;
    const double* r1 = J1 + (size_t)tp[1] * W;
    int64_t rot = (int64_t)sign * (t - tp[1]);
    for (int32_t x = 0; x < W; x++) J[(size_t)t * W + x] = r0[x] + r1[imod(x + rot, W)];
  }
  free(J0);
  free(J1);
}

/* Adjoint of one cyclic transform: the exact transpose of Algorithm 1's
 * merge.  J(t) = R0[t0] + Rotate(R1[t1], s) gives gR0[t0] += gJ(t) and
 * gR1[t1][(x + s) mod W] += gJ(t)[x]; then recurse into both halves. */
static void fht_rec_adj_f64(int32_t n, int32_t W, const double* gJ, double* gI, int32_t split, int sign) {
  if (n == 1) {
    memcpy(gI, gJ, sizeof(double) * (size_t)W);
    return;
  }
  int32_t np[2];
  orc_split(n, split, np);
  double* g0 = (double*)calloc((size_t)np[0] * W, sizeof(double));
  double* g1 = (double*)calloc((size_t)np[1] * W, sizeof(double));
  for (int32_t t = 0; t < n; t++) {
    int32_t tp[2];
    child_slopes(n, np, t, tp);
    int64_t rot = (int64_t)sign * (t - tp[1]);
    for (int32_t x = 0; x < W; x++) {
      double g = gJ[(size_t)t * W + x];
      g0[(size_t)tp[0] * W + x] += g;
      g1[(size_t)tp[1] * W + imod(x + rot, W)] += g;
    }
  }
  fht_rec_adj_f64(np[0], W, g0, gI, split, sign);
  fht_rec_adj_f64(np[1], W, g1, gI + (size_t)np[0] * W, split, sign);
  free(g0);
  free(g1);
}

/* ---------------------------------------------------------------------- */
/* Quadrant views.  Quadrant q of an h x w image:                          */
/*   q = 0, 1: the image itself (n = h split rows, row length w);          */
/*   q = 2, 3: the transposed image (n = w, row length h).                 */
/* Row length W of the view: the real length L (CYCLIC) or L + n - 1       */
/* (EXTENDED, zero padding on the right).  sign = +1 for q = 0, 2.         */
/* ---------------------------------------------------------------------- */
static void view_dims(int32_t h, int32_t w, int q, int boundary, int32_t* n, int32_t* L, int32_t* W) {
  if (q < 2) {
    *n = h;
    *L = w;
  } else {
    *n = w;
    *L = h;
  }
  *W = boundary == ORC_EXTENDED ? *L + *n - 1 : *L;
}

int64_t orc_out_elems(int32_t h, int32_t w, uint32_t quads, int32_t boundary) {
  int64_t total = 0;
  for (int q = 0; q < 4; q++) {
    if (!(quads & (1u << q))) continue;
    int32_t n, L, W;
    view_dims(h, w, q, boundary, &n, &L, &W);
    total += (int64_t)n * W;
  }
  return total;
}

static int64_t* view_i64(const int64_t* img, int32_t h, int32_t w, int q, int32_t n, int32_t W) {
  int64_t* v = (int64_t*)calloc((size_t)n * W, sizeof(int64_t));
  for (int32_t y = 0; y < h; y++)
    for (int32_t x = 0; x < w; x++) {
      if (q < 2)
        v[(size_t)y * W + x] = img[(size_t)y * w + x];
      else
        v[(size_t)x * W + y] = img[(size_t)y * w + x];
    }
  return v;
}

static double* view_f64(const double* img, int32_t h, int32_t w, int q, int32_t n, int32_t W) {
  double* v = (double*)calloc((size_t)n * W, sizeof(double));
  for (int32_t y = 0; y < h; y++)
    for (int32_t x = 0; x < w; x++) {
      if (q < 2)
        v[(size_t)y * W + x] = img[(size_t)y * w + x];
      else
        v[(size_t)x * W + y] = img[(size_t)y * w + x];
    }
  return v;
}

/* O1: the recursion.  out holds the requested quadrants packed in order
 * Q0..Q3, each an n x W row-major block. */
void orc_fht_i64(int32_t h, int32_t w, const int64_t* img, uint32_t quads, int32_t boundary, int32_t split,
                 int64_t* out) {
  for (int q = 0; q < 4; q++) {
    if (!(quads & (1u << q))) continue;
    int32_t n, L, W;
    view_dims(h, w, q, boundary, &n, &L, &W);
    int64_t* v = view_i64(img, h, w, q, n, W);
    fht_rec_i64(n, W, v, out, split, (q & 1) ? -1 : 1);
    free(v);
    out += (size_t)n * W;
  }
}

void orc_fht_f64(int32_t h, int32_t w, const double* img, uint32_t quads, int32_t boundary, int32_t split,
                 double* out) {
  for (int q = 0; q < 4; q++) {
    if (!(quads & (1u << q))) continue;
    int32_t n, L, W;
    view_dims(h, w, q, boundary, &n, &L, &W);
    double* v = view_f64(img, h, w, q, n, W);
    fht_rec_f64(n, W, v, out, split, (q & 1) ? -1 : 1);
    free(v);
    out += (size_t)n * W;
  }
}

/* O2: brute force.  Every pattern is built by Algorithm 2 and the image is
 * summed along it pixel by pixel:  H[t][x] = sum_y V[y][(x + sign pat(y)) mod W]. */
void orc_brute_i64(int32_t h, int32_t w, const int64_t* img, uint32_t quads, int32_t boundary, int32_t split,
                   int64_t* out) {
  for (int q = 0; q < 4; q++) {
    if (!(quads & (1u << q))) continue;
    int32_t n, L, W;
    view_dims(h, w, q, boundary, &n, &L, &W);
    int64_t* v = view_i64(img, h, w, q, n, W);
    int32_t* pat = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int sign = (q & 1) ? -1 : 1;
    for (int32_t t = 0; t < n; t++) {
      orc_pattern(n, t, split, pat);
      for (int32_t x = 0; x < W; x++) {
        int64_t acc = 0;
        for (int32_t y = 0; y < n; y++) acc += v[(size_t)y * W + imod((int64_t)x + sign * pat[y], W)];
        out[(size_t)t * W + x] = acc;
      }
    }
    free(pat);
    free(v);
    out += (size_t)n * W;
  }
}

void orc_brute_f64(int32_t h, int32_t w, const double* img, uint32_t quads, int32_t boundary, int32_t split,
                   double* out) {
  for (int q = 0; q < 4; q++) {
    if (!(quads & (1u << q))) continue;
    int32_t n, L, W;
    view_dims(h, w, q, boundary, &n, &L, &W);
    double* v = view_f64(img, h, w, q, n, W);
    int32_t* pat = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int sign = (q & 1) ? -1 : 1;
    for (int32_t t = 0; t < n; t++) {
      orc_pattern(n, t, split, pat);
      for (int32_t x = 0; x < W; x++) {
        double acc = 0;
        for (int32_t y = 0; y < n; y++) acc += v[(size_t)y * W + imod((int64_t)x + sign * pat[y], W)];
        out[(size_t)t * W + x] = acc;
      }
    }
    free(pat);
    free(v);
    out += (size_t)n * W;
  }
}

/* Adjoint (back-projection) of the packed multi-quadrant transform, by the
 * transposed recursion: gimg = sum over quadrants of Q^T(gout_q), restricted
 * to the real h x w pixels (the padding columns carry no input). */
void orc_adjoint_f64(int32_t h, int32_t w, const double* gout, uint32_t quads, int32_t boundary, int32_t split,
                     double* gimg) {
  memset(gimg, 0, sizeof(double) * (size_t)h * w);
  for (int q = 0; q < 4; q++) {
    if (!(quads & (1u << q))) continue;
    int32_t n, L, W;
    view_dims(h, w, q, boundary, &n, &L, &W);
    double* gv = (double*)malloc(sizeof(double) * (size_t)n * W);
    fht_rec_adj_f64(n, W, gout, gv, split, (q & 1) ? -1 : 1);
    for (int32_t y = 0; y < h; y++)
      for (int32_t x = 0; x < w; x++)
        gimg[(size_t)y * w + x] += (q < 2) ? gv[(size_t)y * W + x] : gv[(size_t)x * W + y];
    free(gv);
    gout += (size_t)n * W;
  }
}

/* Adjoint by brute force: every pattern scatters its Hough value back onto
 * the pixels it sums. */
void orc_adjoint_brute_f64(int32_t h, int32_t w, const double* gout, uint32_t quads, int32_t boundary,
                           int32_t split, double* gimg) {
  memset(gimg, 0, sizeof(double) * (size_t)h * w);
  for (int q = 0; q < 4; q++) {
    if (!(quads & (1u << q))) continue;
    int32_t n, L, W;
    view_dims(h, w, q, boundary, &n, &L, &W);
    int32_t* pat = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int sign = (q & 1) ? -1 : 1;
    for (int32_t t = 0; t < n; t++) {
      orc_pattern(n, t, split, pat);
      for (int32_t x = 0; x < W; x++) {
        double g = gout[(size_t)t * W + x];
        for (int32_t y = 0; y < n; y++) {
          int32_t c = imod((int64_t)x + sign * pat[y], W);
          if (c >= L) continue; /* padding column */
          if (q < 2)
            gimg[(size_t)y * w + c] += g;
          else
            gimg[(size_t)c * w + y] += g;
        }
      }
    }
    free(pat);
    gout += (size_t)n * W;
  }
}

/* ---------------------------------------------------------------------- */
/* The classical Brady-Yong transform for n = 2^q rows (Section 2; the     */
/* paper states that both variants reduce to it for powers of two).        */
/* Written separately from Algorithm 1: bottom-up over block sizes, with   */
/* the classical rule that a line of total displacement d in a block of    */
/* 2b rows is the displacement-floor(d/2) line of the upper b rows plus    */
/* the displacement-floor(d/2) line of the lower b rows started            */
/* ceil(d/2) columns further on.  No rounding function is involved.        */
/* Returns -1 when n is not a power of two.                                 */
/* ---------------------------------------------------------------------- */
int orc_brady_yong_i64(int32_t n, int32_t W, const int64_t* img, int64_t* out) {
  if (n < 1 || (n & (n - 1))) return -1;
  int64_t* a = (int64_t*)malloc(sizeof(int64_t) * (size_t)n * W);
  int64_t* b = (int64_t*)malloc(sizeof(int64_t) * (size_t)n * W);
  memcpy(a, img, sizeof(int64_t) * (size_t)n * W);
  for (int32_t bs = 1; bs < n; bs *= 2) {
    /* merge pairs of bs-row blocks into 2bs-row blocks */
    for (int32_t base = 0; base < n; base += 2 * bs) {
      for (int32_t d = 0; d < 2 * bs; d++) {
        const int64_t* up = a + (size_t)(base + d / 2) * W;
        const int64_t* lo = a + (size_t)(base + bs + d / 2) * W;
        int32_t off = (d + 1) / 2;
        int64_t* o = b + (size_t)(base + d) * W;
        for (int32_t x = 0; x < W; x++) o[x] = up[x] + lo[(x + off) % W];
      }
    }
    int64_t* tmp = a;
    a = b;
    b = tmp;
  }
  memcpy(out, a, sizeof(int64_t) * (size_t)n * W);
  free(a);
  free(b);
  return 0;
}

/* Sampled brute force: the definition evaluated at chosen outputs only.
 * For sample k (quadrant q[k], slope t[k], output column x[k]):
 *   val[k]  = sum_y V[y][(x + sign pat(n,t)[y]) mod W]       (the Hough value)
 *   mass[k] = sum_y |V[y][(x + sign pat(n,t)[y]) mod W]|     (the pattern's L1 mass)
 * V is the quadrant's view of the image (transposed for q >= 2), zero outside
 * the real columns.  Used for full-size images where O1 would be too slow. */
void orc_brute_at_f64(int32_t h, int32_t w, const double* img, int32_t boundary, int32_t split, int64_t nsamp,
                      const int32_t* qs, const int32_t* ts, const int32_t* xs, double* val, double* mass) {
  int32_t* pat = (int32_t*)malloc(sizeof(int32_t) * (size_t)(h > w ? h : w));
  for (int64_t k = 0; k < nsamp; k++) {
    int q = qs[k];
    int32_t n, L, W;
    view_dims(h, w, q, boundary, &n, &L, &W);
    int sign = (q & 1) ? -1 : 1;
    orc_pattern(n, ts[k], split, pat);
    double acc = 0, m = 0;
    for (int32_t y = 0; y < n; y++) {
      int32_t c = imod((int64_t)xs[k] + sign * pat[y], W);
      if (c >= L) continue;
      double v = (q < 2) ? img[(size_t)y * w + c] : img[(size_t)c * w + y];
      acc += v;
      m += v < 0 ? -v : v;
    }
    val[k] = acc;
    mass[k] = m;
  }
  free(pat);
}

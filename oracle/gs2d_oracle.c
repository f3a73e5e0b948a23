/*
 * gs2d oracle -- plain, slow, brute-force CPU reference for the 2D Gaussian
 * rasterizer of "Neural Video Compression using 2D Gaussian Splatting"
 * (arXiv 2505.09324).  TEST INFRASTRUCTURE ONLY: the product path never links
 * or calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or constant table with the CUDA
 * library.
 *
 * What it computes (all in double precision unless stated):
 *
 *   Gaussian n (Sec. 3.1): mean mu = (mx, my), Cholesky vector l = (l1, l2, l3)
 *   with L = [[l1, 0], [l2, l3]] and covariance Sigma = L L^T (Eq. 1), colour
 *   c = (cr, cg, cb), weight w (the colour coefficient of Eq. 2 is c' = w c).
 *
 *   Accumulated-sum blending (Eq. 2): for pixel (x, y) with centre
 *   p = (x + 0.5, y + 0.5),
 *        C(p) = sum_n  c_n * w_n * exp(-sigma_n(p)),
 *        sigma_n(p) = 1/2 (p - mu_n)^T Sigma_n^{-1} (p - mu_n),
 *   summed over the Gaussians that "contribute" at p, in ascending n.  The
 *   paper leaves sigma_n undefined and gives no cut-off; the readings used here
 *   (the half Mahalanobis form and the predicate below) are project readings.
 *
 *   Contribution predicate: all nine parameters finite, det Sigma > det_eps,
 *   and sigma_n(p) <= tau_n with tau_n = min(sigma_cut, ln(|w_n| / alpha_min)).
 *
 *   Loss (L2): L = 1/(3HW) sum (C - T)^2, dL/dC = 2 (C - T) / (3HW).
 *
 *   Gradients by matrix calculus on the plain definition (Sec. 3.1 optimises the
 *   factorised form): with Q = Sigma^{-1}, d = p - mu, alpha = w exp(-sigma),
 *   s = dL/dsigma = -(g . c) alpha:
 *        dL/dc    = sum g alpha            dL/dw = sum (g . c) exp(-sigma)
 *        dL/dmu   = sum s * (-Q d)         dL/dQ = sum s * (1/2) d d^T
 *        dL/dSigma = -Q (dL/dQ) Q          dL/dL = 2 (dL/dSigma) L  (lower part).
 *
 *   Tile binning (the "tile-based rasterization" the method inherits, Sec. 3):
 *   computed in single precision with exactly these single-rounded operations
 *   (the file is compiled with -ffp-contract=off so no FMA is formed):
 *        Sxx = l1*l1, Syy = l2*l2 + l3*l3, a = l1*l3, det = a*a,
 *        k = sqrt(2*sigma_cut), rx = ceil(k * sqrt(Sxx)), ry = ceil(k * sqrt(Syy))
 *        (the axis-aligned box of the sigma <= sigma_cut ellipse; k = 3 at
 *        sigma_cut = 4.5),
 *        px0 = floor(mx - rx), px1 = floor(mx + rx)  (same in y with ry),
 *   clipped to the image; tiles tx0 = xlo / T .. xhi / T inclusive.  A Gaussian
 *   is culled when a parameter is non-finite, det <= det_eps, |w| < alpha_min
 *   or its clipped rectangle is empty.  The key of a (tile, n) pair is
 *   tile * 2^32 + n; keys are unique, so their sorted order is unique.
 *
 * Ambiguity bookkeeping: the FP32 GPU path evaluates the predicate in single
 * precision, so a pair whose sigma lies within amb_tol * max(1, tau) of tau may
 * legitimately go either way.  Such pairs are not added to the definite result;
 * their contribution is reported separately (as [lo, hi] bounds for the image,
 * as an absolute-value bound for gradients) so a test can accept either choice.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

typedef struct {
  double sigma_cut; /* cut-off on sigma (4.5: the 3-sigma ellipse) */
  double alpha_min; /* minimum |alpha| (1/255) */
  double det_eps;   /* minimum det Sigma */
  double amb_tol;   /* ambiguity band, relative to max(1, tau) */
} orc_cfg;

/* ------------------------------------------------------------------ */
/* one Gaussian in double precision, built from the plain definition    */

typedef struct {
  int active;
  double mx, my, l1, l2, l3, c[3], w;
  double sxx, sxy, syy, det;
  double qxx, qxy, qyy; /* Q = Sigma^{-1} */
  double tau;
  double hx, hy; /* half extents of the sigma <= sigma_cut ellipse */
} orc_gauss;

static int all_finite(const double* v, int k) {
  for (int i = 0; i < k; i++)
    if (!isfinite(v[i])) return 0;
  return 1;
}

static void orc_load(const double* p, int n, int i, const orc_cfg* cfg, orc_gauss* g) {
  double v[9];
  for (int r = 0; r < 9; r++) v[r] = p[(size_t)r * n + i];
  memset(g, 0, sizeof(*g));
  g->mx = v[0];
  g->my = v[1];
  g->l1 = v[2];
  g->l2 = v[3];
  g->l3 = v[4];
  g->c[0] = v[5];
  g->c[1] = v[6];
  g->c[2] = v[7];
  g->w = v[8];
  if (!all_finite(v, 9)) return;
  /* Sigma = L L^T with L = [[l1, 0], [l2, l3]] (Eq. 1) */
  g->sxx = g->l1 * g->l1;
  g->sxy = g->l1 * g->l2;
  g->syy = g->l2 * g->l2 + g->l3 * g->l3;
  g->det = g->sxx * g->syy - g->sxy * g->sxy;
  if (!(g->det > cfg->det_eps)) return;
  g->qxx = g->syy / g->det;
  g->qxy = -g->sxy / g->det;
  g->qyy = g->sxx / g->det;
  if (g->w == 0.0) return;
  g->tau = log(fabs(g->w) / cfg->alpha_min);
  if (g->tau > cfg->sigma_cut) g->tau = cfg->sigma_cut;
  /* sigma <= s_cut  <=>  d^T Q d <= 2 s_cut: half extent sqrt(2 s_cut Sxx) */
  g->hx = sqrt(2.0 * cfg->sigma_cut * g->sxx);
  g->hy = sqrt(2.0 * cfg->sigma_cut * g->syy);
  /* tau < 0 admits no pixel (sigma >= 0) except inside the ambiguity band */
  g->active = g->tau >= -cfg->amb_tol;
}

static double orc_sigma(const orc_gauss* g, double px, double py) {
  double dx = px - g->mx, dy = py - g->my;
  return 0.5 * (g->qxx * dx * dx + 2.0 * g->qxy * dx * dy + g->qyy * dy * dy);
}

/* 0: no contribution, 1: definite contribution, 2: ambiguous */
static int orc_classify(const orc_gauss* g, double sigma, const orc_cfg* cfg) {
  double band = cfg->amb_tol * (g->tau > 1.0 ? g->tau : 1.0);
  if (fabs(sigma - g->tau) <= band) return 2;
  return sigma <= g->tau ? 1 : 0;
}

/* pixel range [lo, hi] of a Gaussian along one axis for the "fast" mode:
 * every pixel centre within the ellipse half extent h (plus one pixel of slack) */
static void orc_span(double m, double h, int size, int* lo, int* hi) {
  double a = floor(m - h - 1.0), b = ceil(m + h + 1.0);
  if (a < 0) a = 0;
  if (a > size) a = size;
  if (b > size - 1) b = size - 1;
  if (b < -1) b = -1;
  *lo = (int)a;
  *hi = (int)b;
}

/*
 * Forward render (Eq. 2).  img: [3][H][W] definite sum.  amb_lo / amb_hi
 * (nullable): per-channel sums of the negative / positive parts of ambiguous
 * contributions.  fast != 0 restricts each Gaussian to its ellipse bounding box
 * (exact, because a pair outside it has sigma > sigma_cut >= tau); fast == 0 is
 * the brute force over every (pixel, Gaussian) pair.
 */
int orc_render(int W, int H, int n, const double* p, const orc_cfg* cfg, int fast,
               double* img, double* amb_lo, double* amb_hi) {
  if (W < 0 || H < 0 || n < 0 || !cfg || !img) return ORC_EINVAL;
  orc_gauss* gs = (orc_gauss*)malloc(sizeof(orc_gauss) * (n > 0 ? n : 1));
  if (!gs) return ORC_ENOMEM;
  for (int i = 0; i < n; i++) orc_load(p, n, i, cfg, &gs[i]);
  const size_t HW = (size_t)H * W;
#pragma omp parallel for schedule(dynamic, 1)
  for (int y = 0; y < H; y++) {
    double py = y + 0.5;
    for (int x = 0; x < W; x++) {
      size_t o = (size_t)y * W + x;
      for (int ch = 0; ch < 3; ch++) {
        img[ch * HW + o] = 0.0;
        if (amb_lo) amb_lo[ch * HW + o] = 0.0;
        if (amb_hi) amb_hi[ch * HW + o] = 0.0;
      }
    }
    for (int i = 0; i < n; i++) {
      const orc_gauss* g = &gs[i];
      if (!g->active) continue;
      int x0 = 0, x1 = W - 1;
      if (fast) {
        int ylo, yhi;
        orc_span(g->my, g->hy, H, &ylo, &yhi);
        if (y < ylo || y > yhi) continue;
        orc_span(g->mx, g->hx, W, &x0, &x1);
      }
      for (int x = x0; x <= x1; x++) {
        double s = orc_sigma(g, x + 0.5, py);
        int k = orc_classify(g, s, cfg);
        if (k == 0) continue;
        double alpha = g->w * exp(-s);
        size_t o = (size_t)y * W + x;
        for (int ch = 0; ch < 3; ch++) {
          double v = g->c[ch] * alpha;
          if (k == 1) {
            img[ch * HW + o] += v;
          } else if (v < 0) {
            if (amb_lo) amb_lo[ch * HW + o] += v;
          } else {
            if (amb_hi) amb_hi[ch * HW + o] += v;
          }
        }
      }
    }
  }
  free(gs);
  return ORC_OK;
}

/* Render only the listed pixels (xy: [npix][2] integer pixel coordinates). */
int orc_render_pixels(int n, const double* p, const orc_cfg* cfg, int npix, const int32_t* xy,
                      double* out /*[3][npix]*/, double* amb_lo, double* amb_hi) {
  if (n < 0 || npix < 0 || !cfg || !out) return ORC_EINVAL;
  orc_gauss* gs = (orc_gauss*)malloc(sizeof(orc_gauss) * (n > 0 ? n : 1));
  if (!gs) return ORC_ENOMEM;
  for (int i = 0; i < n; i++) orc_load(p, n, i, cfg, &gs[i]);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < npix; k++) {
    double px = xy[2 * k] + 0.5, py = xy[2 * k + 1] + 0.5;
    double acc[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int i = 0; i < n; i++) {
      const orc_gauss* g = &gs[i];
      if (!g->active) continue;
      double s = orc_sigma(g, px, py);
      int c = orc_classify(g, s, cfg);
      if (c == 0) continue;
      double alpha = g->w * exp(-s);
      for (int ch = 0; ch < 3; ch++) {
        double v = g->c[ch] * alpha;
        if (c == 1)
          acc[ch] += v;
        else if (v < 0)
          lo[ch] += v;
        else
          hi[ch] += v;
      }
    }
    for (int ch = 0; ch < 3; ch++) {
      out[(size_t)ch * npix + k] = acc[ch];
      if (amb_lo) amb_lo[(size_t)ch * npix + k] = lo[ch];
      if (amb_hi) amb_hi[(size_t)ch * npix + k] = hi[ch];
    }
  }
  free(gs);
  return ORC_OK;
}

/*
 * Backward: gradients of L with respect to the nine parameters of each Gaussian
 * given g = dL/dC ([3][H][W]).  grad: [9][n] (rows mx, my, l1, l2, l3, cr, cg,
 * cb, w).  Optional g_unc ([3][H][W], >= 0): an uncertainty bound on g; grad_unc
 * ([9][n], nullable) then receives sum |partial| over ambiguous pairs plus
 * sum g_unc * |dC/dtheta| over definite pairs, a first-order bound on how far a
 * correct single-precision implementation may lie from grad.
 * which (nullable, nwhich entries): compute only these Gaussians (others 0).
 */
int orc_render_grad(int W, int H, int n, const double* p, const orc_cfg* cfg, int fast,
                    const double* g, const double* g_unc, const int32_t* which, int nwhich,
                    double* grad, double* grad_unc) {
  if (W < 0 || H < 0 || n < 0 || !cfg || !g || !grad) return ORC_EINVAL;
  memset(grad, 0, sizeof(double) * 9 * (size_t)n);
  if (grad_unc) memset(grad_unc, 0, sizeof(double) * 9 * (size_t)n);
  const size_t HW = (size_t)H * W;
  int count = which ? nwhich : n;
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k < count; k++) {
    int i = which ? which[k] : k;
    if (i < 0 || i >= n) continue;
    orc_gauss G;
    orc_load(p, n, i, cfg, &G);
    if (!G.active) continue;
    int x0 = 0, x1 = W - 1, y0 = 0, y1 = H - 1;
    if (fast) {
      orc_span(G.mx, G.hx, W, &x0, &x1);
      orc_span(G.my, G.hy, H, &y0, &y1);
    }
    /* accumulators: dc[3], dw, s*d (2), s*d d^T / 2 (xx, xy, yy) and the
     * matching absolute-value sums for the uncertainty bound */
    double dc[3] = {0, 0, 0}, dw = 0, sd[2] = {0, 0}, sdd[3] = {0, 0, 0};
    double uc[3] = {0, 0, 0}, uw = 0, usd[2] = {0, 0}, usdd[3] = {0, 0, 0};
    for (int y = y0; y <= y1; y++) {
      double py = y + 0.5;
      for (int x = x0; x <= x1; x++) {
        double px = x + 0.5;
        double sg = orc_sigma(&G, px, py);
        int cls = orc_classify(&G, sg, cfg);
        if (cls == 0) continue;
        size_t o = (size_t)y * W + x;
        double e = exp(-sg), alpha = G.w * e;
        double gv[3] = {g[o], g[HW + o], g[2 * HW + o]};
        double gc = gv[0] * G.c[0] + gv[1] * G.c[1] + gv[2] * G.c[2];
        double s = -gc * alpha; /* dL/dsigma */
        double dx = px - G.mx, dy = py - G.my;
        if (cls == 1) {
          for (int ch = 0; ch < 3; ch++) dc[ch] += gv[ch] * alpha;
          dw += gc * e;
          sd[0] += s * dx;
          sd[1] += s * dy;
          sdd[0] += 0.5 * s * dx * dx;
          sdd[1] += 0.5 * s * dx * dy;
          sdd[2] += 0.5 * s * dy * dy;
          if (g_unc && grad_unc) {
            double gu[3] = {g_unc[o], g_unc[HW + o], g_unc[2 * HW + o]};
            double guc = gu[0] * fabs(G.c[0]) + gu[1] * fabs(G.c[1]) + gu[2] * fabs(G.c[2]);
            double su = guc * fabs(alpha);
            for (int ch = 0; ch < 3; ch++) uc[ch] += gu[ch] * fabs(alpha);
            uw += guc * e;
            usd[0] += su * fabs(dx);
            usd[1] += su * fabs(dy);
            usdd[0] += 0.5 * su * dx * dx;
            usdd[1] += 0.5 * su * fabs(dx * dy);
            usdd[2] += 0.5 * su * dy * dy;
          }
        } else {
          for (int ch = 0; ch < 3; ch++) uc[ch] += fabs(gv[ch] * alpha);
          uw += fabs(gc * e);
          usd[0] += fabs(s * dx);
          usd[1] += fabs(s * dy);
          usdd[0] += 0.5 * fabs(s) * dx * dx;
          usdd[1] += 0.5 * fabs(s * dx * dy);
          usdd[2] += 0.5 * fabs(s) * dy * dy;
        }
      }
    }
    /* dL/dmu = -Q (sum s d) */
    double gmx = -(G.qxx * sd[0] + G.qxy * sd[1]);
    double gmy = -(G.qxy * sd[0] + G.qyy * sd[1]);
    /* dL/dQ = [[sdd0, sdd1], [sdd1, sdd2]];  dL/dSigma = -Q dLdQ Q */
    double A[2][2] = {{sdd[0], sdd[1]}, {sdd[1], sdd[2]}};
    double Q[2][2] = {{G.qxx, G.qxy}, {G.qxy, G.qyy}};
    double T1[2][2], GS[2][2];
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++) T1[a][b] = Q[a][0] * A[0][b] + Q[a][1] * A[1][b];
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++) GS[a][b] = -(T1[a][0] * Q[0][b] + T1[a][1] * Q[1][b]);
    /* dL/dL = 2 GS L, L = [[l1, 0], [l2, l3]] -> entries (0,0), (1,0), (1,1) */
    double Lm[2][2] = {{G.l1, 0.0}, {G.l2, G.l3}};
    double dL[2][2];
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++) dL[a][b] = 2.0 * (GS[a][0] * Lm[0][b] + GS[a][1] * Lm[1][b]);
    /* dL/dc_ch = sum g_ch alpha (alpha already contains w) */
    double out[9] = {gmx, gmy, dL[0][0], dL[1][0], dL[1][1], dc[0], dc[1], dc[2], dw};
    for (int r = 0; r < 9; r++) grad[(size_t)r * n + i] = out[r];
    if (grad_unc) {
      /* propagate the absolute sums through the same linear maps with |.| */
      double aQ[2][2] = {{fabs(G.qxx), fabs(G.qxy)}, {fabs(G.qxy), fabs(G.qyy)}};
      double uA[2][2] = {{usdd[0], usdd[1]}, {usdd[1], usdd[2]}};
      double uT[2][2], uG[2][2], uL[2][2];
      double aLm[2][2] = {{fabs(G.l1), 0.0}, {fabs(G.l2), fabs(G.l3)}};
      for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) uT[a][b] = aQ[a][0] * uA[0][b] + aQ[a][1] * uA[1][b];
      for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) uG[a][b] = uT[a][0] * aQ[0][b] + uT[a][1] * aQ[1][b];
      for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) uL[a][b] = 2.0 * (uG[a][0] * aLm[0][b] + uG[a][1] * aLm[1][b]);
      double u[9] = {aQ[0][0] * usd[0] + aQ[0][1] * usd[1], aQ[1][0] * usd[0] + aQ[1][1] * usd[1],
                     uL[0][0], uL[1][0], uL[1][1], uc[0], uc[1], uc[2], uw};
      for (int r = 0; r < 9; r++) grad_unc[(size_t)r * n + i] = u[r];
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* tile binning in single precision                                      */

/* Per-Gaussian tile rectangle [tx0, tx1) x [ty0, ty1) and tile count. */
static int orc_rect32(int W, int H, int T, float mx, float my, float l1, float l2, float l3,
                      float cr, float cg, float cb, float w, float sigma_cut, float alpha_min,
                      float det_eps, int32_t rect[4]) {
  rect[0] = rect[1] = rect[2] = rect[3] = 0;
  if (!(isfinite(mx) && isfinite(my) && isfinite(l1) && isfinite(l2) && isfinite(l3) &&
        isfinite(cr) && isfinite(cg) && isfinite(cb) && isfinite(w)))
    return 0;
  float sxx = l1 * l1;
  float t1 = l2 * l2;
  float t2 = l3 * l3;
  float syy = t1 + t2;
  float a = l1 * l3;
  float det = a * a;
  if (!(det > det_eps)) return 0;
  if (!(fabsf(w) >= alpha_min)) return 0;
  /* the sigma <= sigma_cut ellipse {d : d^T Sigma^-1 d <= 2 sigma_cut} reaches
   * sqrt(2 sigma_cut Sxx) along x and sqrt(2 sigma_cut Syy) along y; at
   * sigma_cut = 4.5 the factor is exactly 3 */
  float kc = sqrtf(2.0f * sigma_cut);
  float rx = ceilf(kc * sqrtf(sxx));
  float ry = ceilf(kc * sqrtf(syy));
  float fx0 = floorf(mx - rx), fx1 = floorf(mx + rx);
  float fy0 = floorf(my - ry), fy1 = floorf(my + ry);
  /* clip to the image (as floats first so huge values cannot overflow int) */
  if (fx0 < 0.0f) fx0 = 0.0f;
  if (fy0 < 0.0f) fy0 = 0.0f;
  if (fx1 > (float)(W - 1)) fx1 = (float)(W - 1);
  if (fy1 > (float)(H - 1)) fy1 = (float)(H - 1);
  if (fx0 > fx1 || fy0 > fy1) return 0;
  int x0 = (int)fx0, x1 = (int)fx1, y0 = (int)fy0, y1 = (int)fy1;
  rect[0] = x0 / T;
  rect[1] = y0 / T;
  rect[2] = x1 / T + 1;
  rect[3] = y1 / T + 1;
  return (rect[2] - rect[0]) * (rect[3] - rect[1]);
}

/* rect: [n][4] (tx0, ty0, tx1, ty1), count: [n]; returns total entries via *total */
int orc_tile_rects(int W, int H, int T, int n, const float* p, float sigma_cut, float alpha_min,
                   float det_eps, int32_t* rect, int32_t* count, int64_t* total) {
  if (W <= 0 || H <= 0 || T <= 0 || n < 0 || !rect || !count || !total) return ORC_EINVAL;
  int64_t tot = 0;
  for (int i = 0; i < n; i++) {
    const size_t m = (size_t)n;
    count[i] = orc_rect32(W, H, T, p[i], p[m + i], p[2 * m + i], p[3 * m + i], p[4 * m + i],
                          p[5 * m + i], p[6 * m + i], p[7 * m + i], p[8 * m + i], sigma_cut,
                          alpha_min, det_eps, &rect[4 * (size_t)i]);
    tot += count[i];
  }
  *total = tot;
  return ORC_OK;
}

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/*
 * All (tile, n) keys sorted ascending (key = tile << 32 | n), and per-tile
 * ranges [start, end) into the sorted list.  keys must hold `total` entries as
 * returned by orc_tile_rects; ranges: [TX*TY][2].
 */
int orc_sorted_keys(int W, int H, int T, int n, const int32_t* rect, int64_t total,
                    uint64_t* keys, int32_t* ranges) {
  if (W <= 0 || H <= 0 || T <= 0 || n < 0 || !rect || (!keys && total > 0) || !ranges)
    return ORC_EINVAL;
  int TX = (W + T - 1) / T, TY = (H + T - 1) / T;
  int64_t k = 0;
  for (int i = 0; i < n; i++) {
    const int32_t* r = &rect[4 * (size_t)i];
    for (int ty = r[1]; ty < r[3]; ty++)
      for (int tx = r[0]; tx < r[2]; tx++) {
        if (k >= total) return ORC_EINVAL;
        keys[k++] = ((uint64_t)(uint32_t)(ty * TX + tx) << 32) | (uint32_t)i;
      }
  }
  if (k != total) return ORC_EINVAL;
  qsort(keys, (size_t)total, sizeof(uint64_t), cmp_u64);
  for (int t = 0; t < TX * TY; t++) ranges[2 * t] = ranges[2 * t + 1] = 0;
  for (int64_t j = 0; j < total; j++) {
    int t = (int)(keys[j] >> 32);
    if (j == 0 || (int)(keys[j - 1] >> 32) != t) ranges[2 * t] = (int32_t)j;
    ranges[2 * t + 1] = (int32_t)(j + 1);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* thread control for timing the oracle on a stated number of cores     */
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_set_threads(int k) {
#ifdef _OPENMP
  if (k > 0) omp_set_num_threads(k);
  return omp_get_max_threads();
#else
  (void)k;
  return 1;
#endif
}

/*
 * CPU oracle for geodesic 3x3 chains. TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline and
 * reference legs call this code. It shares nothing with the CUDA library (no header, no helper, no
 * constant) and is written as the plain definitions from Zlaus & Mongus,
 * "Efficient method for parallel computation of geodesic transformation on
 * CPU" (IEEE TPDS 2019):
 *
 *   Section 2, Eq. 1-2  erosion / dilation by the square w_s(p), which is
 *                       clipped to the image domain P (w_s(p) is a subset of P)
 *   Section 2, Eq. 3    elementary geodesic erosion  max(eps_1(f), m)
 *                       and its dual dilation        min(delta_1(f), m)
 *   Section 2, Eq. 4    geodesic erosion/dilation of size s = s nested steps
 *   Section 2, Eq. 5    reconstruction = the limit of the chain (iterate until
 *                       a step changes nothing, as in Section 3.7, Algorithm 5)
 *   Section 2, Eq. 6-12 geodesic operators built on reconstruction
 *   Section 2, Eq. 13-15 quasi-distance transform (residuals of an erosion
 *                       chain as in Algorithm 6, then the eta iteration)
 *   Section 2, Eq. 16-20 openings, closings, granulometric function, pattern
 *                       spectrum and alternating sequential filters
 *
 * Every value is held as a double. uint8 and float32 images convert to double
 * exactly, and the forward operators only select among their inputs, so the
 * results convert back exactly. The backward pass (not in the paper) sums
 * upstream gradients in double.
 *
 * Images are row-major, contiguous, H rows of W pixels; index y * W + x.
 * conn = 8 uses the 3x3 square w_1; conn = 4 uses the cross (centre plus
 * the four edge neighbours), which the paper does not use; it is this
 * library's extension. Pixels outside the image are skipped, never padded.
 */
#include <stdlib.h>
#include <string.h>

enum { ORA_DILATE = 0, ORA_ERODE = 1 };

/* neighbour k = (dy + 1) * 3 + (dx + 1); the cross keeps k in {1, 3, 4, 5, 7} */
static int ora_in_shape(int conn, int dy, int dx)
{
    return conn == 8 || dy == 0 || dx == 0;
}

/* extreme of f over the clipped neighbourhood of (y, x): Eq. 1 (op = erode) or
 * Eq. 2 (op = dilate) with s = 1; *k_out gets the lowest neighbour index k
 * that attains it. */
static double ora_extreme(const double *f, long H, long W, int conn, int op,
                          long y, long x, int *k_out)
{
    double best = 0.0;
    int have = 0, bestk = -1;
    for (int dy = -1; dy <= 1; ++dy) {
        for (int dx = -1; dx <= 1; ++dx) {
            if (!ora_in_shape(conn, dy, dx)) continue;
            long qy = y + dy, qx = x + dx;
            if (qy < 0 || qy >= H || qx < 0 || qx >= W) continue;
            double v = f[qy * W + qx];
            int better = !have || (op == ORA_DILATE ? (v > best) : (v < best));
            if (better) {
                best = v;
                bestk = (dy + 1) * 3 + (dx + 1);
                have = 1;
            }
        }
    }
    if (k_out) *k_out = bestk;
    return best;
}

/* One elementary geodesic step (Eq. 3 and its dual). m == NULL: no mask
 * (a plain eps_1 / delta_1 step). Every output pixel depends only on f and
 * m, so the rows are independent: the build with -fopenmp (the benchmark's
 * all-core CPU baseline) splits them over threads; the plain build ignores
 * the pragma. */
void oracle_step(const double *f, const double *m, double *out, long H, long W,
                 int conn, int op)
{
#pragma omp parallel for schedule(static)
    for (long y = 0; y < H; ++y) {
        for (long x = 0; x < W; ++x) {
            double v = ora_extreme(f, H, W, conn, op, y, x, NULL);
            if (m) {
                double mv = m[y * W + x];
                if (op == ORA_DILATE) v = (mv < v) ? mv : v;  /* min(delta_1(f), m) */
                else                  v = (mv > v) ? mv : v;  /* max(eps_1(f), m)   */
            }
            out[y * W + x] = v;
        }
    }
}

/* Geodesic erosion / dilation of size `steps` (Eq. 4): steps nested
 * elementary steps, each computed from the whole previous image. */
int oracle_chain(const double *f, const double *m, double *out, long H, long W,
                 int conn, int op, long steps)
{
    long n = H * W;
    if (n == 0) return 0;
    memcpy(out, f, (size_t)n * sizeof(double));
    if (steps <= 0) return 0;
    double *tmp = (double *)malloc((size_t)n * sizeof(double));
    if (!tmp) return -1;
    for (long s = 0; s < steps; ++s) {
        oracle_step(out, m, tmp, H, W, conn, op);
        memcpy(out, tmp, (size_t)n * sizeof(double));
    }
    free(tmp);
    return 0;
}

/* Reconstruction (Eq. 5): repeat elementary steps until one changes no pixel.
 * Returns the number of steps that changed something, or -1 if max_steps
 * steps all changed something (not converged), or -2 on allocation failure. */
long oracle_reconstruct(const double *f, const double *m, double *out, long H,
                        long W, int conn, int op, long max_steps)
{
    long n = H * W;
    if (n == 0) return 0;
    memcpy(out, f, (size_t)n * sizeof(double));
    double *tmp = (double *)malloc((size_t)n * sizeof(double));
    if (!tmp) return -2;
    long changing = 0;
    for (;;) {
        if (changing >= max_steps) { changing = -1; break; }
        oracle_step(out, m, tmp, H, W, conn, op);
        int changed = 0;
        for (long i = 0; i < n; ++i) {
            if (tmp[i] != out[i]) { changed = 1; break; }
        }
        if (!changed) break;
        memcpy(out, tmp, (size_t)n * sizeof(double));
        ++changing;
    }
    free(tmp);
    return changing;
}

/* Erosion / dilation by the clipped square w_s (Eq. 1-2). The window is the
 * product {x-s..x+s} x {y-s..y+s} intersected with P, so its extreme is the
 * extreme over rows of the extreme over columns; both loops run over the
 * window itself (no running-extreme trick). */
int oracle_window(const double *f, double *out, long H, long W, long s, int op)
{
    long n = H * W;
    if (n == 0) return 0;
    double *row = (double *)malloc((size_t)n * sizeof(double));
    if (!row) return -1;
    for (long y = 0; y < H; ++y) {
        for (long x = 0; x < W; ++x) {
            long x0 = x - s < 0 ? 0 : x - s, x1 = x + s >= W ? W - 1 : x + s;
            double v = f[y * W + x0];
            for (long q = x0 + 1; q <= x1; ++q) {
                double u = f[y * W + q];
                v = (op == ORA_DILATE) ? (u > v ? u : v) : (u < v ? u : v);
            }
            row[y * W + x] = v;
        }
    }
    for (long y = 0; y < H; ++y) {
        long y0 = y - s < 0 ? 0 : y - s, y1 = y + s >= H ? H - 1 : y + s;
        for (long x = 0; x < W; ++x) {
            double v = row[y0 * W + x];
            for (long q = y0 + 1; q <= y1; ++q) {
                double u = row[q * W + x];
                v = (op == ORA_DILATE) ? (u > v ? u : v) : (u < v ? u : v);
            }
            out[y * W + x] = v;
        }
    }
    free(row);
    return 0;
}

/* Reverse mode of the masked chain (Eq. 4), which the paper does not cover.
 *
 * Step t maps f_{t-1} to f_t with f_t(p) = clamp(ext_{q in N(p)} f_{t-1}(q), m(p)).
 * Routing rule at pixel p:
 *   - the mask is selected when it is strictly beyond the neighbourhood
 *     extreme (m(p) < v(p) for dilation, m(p) > v(p) for erosion); the upstream
 *     gradient g_t(p) is then added to grad_mask(p);
 *   - otherwise the gradient goes to the neighbour q = p + d_k, where k is the
 *     lowest neighbour index attaining the extreme.
 * Chain rule as a gather: g_{t-1}(q) = sum over k = 0..8 (in increasing k) of
 * g_t(q - d_k) where pixel q - d_k is in the image and routed to its
 * neighbour k. grad_mask accumulates over t = steps, steps-1, ..., 1.
 * Forward states are all kept in memory. Returns 0, or -1 on allocation
 * failure. */
int oracle_chain_backward(const double *f0, const double *m, const double *gout,
                          double *gmarker, double *gmask, long H, long W,
                          int conn, int op, long steps)
{
    long n = H * W;
    if (n == 0) return 0;
    for (long i = 0; i < n; ++i) gmask[i] = 0.0;
    memcpy(gmarker, gout, (size_t)n * sizeof(double));
    if (steps <= 0) return 0;
    double *states = (double *)malloc((size_t)n * (size_t)steps * sizeof(double));
    double *gnew = (double *)malloc((size_t)n * sizeof(double));
    int *sel = (int *)malloc((size_t)n * sizeof(int));
    if (!states || !gnew || !sel) {
        free(states); free(gnew); free(sel);
        return -1;
    }
    memcpy(states, f0, (size_t)n * sizeof(double));
    for (long t = 1; t < steps; ++t)
        oracle_step(states + (t - 1) * n, m, states + t * n, H, W, conn, op);
    for (long t = steps; t >= 1; --t) {
        const double *fp = states + (t - 1) * n;
        /* routing of step t: sel = neighbour index, or -1 for the mask */
        for (long y = 0; y < H; ++y) {
            for (long x = 0; x < W; ++x) {
                int k;
                double v = ora_extreme(fp, H, W, conn, op, y, x, &k);
                double mv = m[y * W + x];
                int to_mask = (op == ORA_DILATE) ? (mv < v) : (mv > v);
                sel[y * W + x] = to_mask ? -1 : k;
                if (to_mask) gmask[y * W + x] += gmarker[y * W + x];
            }
        }
        for (long y = 0; y < H; ++y) {
            for (long x = 0; x < W; ++x) {
                double acc = 0.0;
                for (int k = 0; k < 9; ++k) {
                    int dy = k / 3 - 1, dx = k % 3 - 1;
                    long py = y - dy, px = x - dx;
                    if (py < 0 || py >= H || px < 0 || px >= W) continue;
                    if (sel[py * W + px] == k) acc += gmarker[py * W + px];
                }
                gnew[y * W + x] = acc;
            }
        }
        memcpy(gmarker, gnew, (size_t)n * sizeof(double));
    }
    free(states); free(gnew); free(sel);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Geodesic operators of Section 2 built on reconstruction (Eq. 6-12).       */
/* ------------------------------------------------------------------------ */

/* Subtraction in the image's element type: the operators below produce
 * pixel values by subtraction (the HMAX marker, DOME, RAOBJ), and a float32
 * image holds the float32-rounded difference. f32 != 0 rounds through float
 * arithmetic; uint8 and float64 differences are exact in double. */
static double ora_sub(double a, double b, int f32)
{
    if (f32) {
        float fa = (float)a, fb = (float)b;
        float d = fa - fb;
        return (double)d;
    }
    return a - b;
}

/* HMAX_h(f) = dilation by reconstruction of f - h under f (Eq. 6). The
 * marker is f - h in the element type, clamped from below by `lo` (0 for
 * uint8 images, -HUGE_VAL otherwise). */
long oracle_hmax(const double *f, double *out, long H, long W, int conn, double h, double lo, int f32)
{
    long n = H * W;
    if (n == 0) return 0;
    double *mk = (double *)malloc((size_t)n * sizeof(double));
    if (!mk) return -2;
    for (long i = 0; i < n; ++i) {
        double d = ora_sub(f[i], h, f32);
        mk[i] = d < lo ? lo : d;
    }
    long r = oracle_reconstruct(mk, f, out, H, W, conn, ORA_DILATE, n + 1);
    free(mk);
    return r;
}

/* DOME_h(f) = f - HMAX_h(f) (Eq. 7). */
long oracle_dome(const double *f, double *out, long H, long W, int conn, double h, double lo, int f32)
{
    long r = oracle_hmax(f, out, H, W, conn, h, lo, f32);
    for (long i = 0; i < H * W; ++i) out[i] = ora_sub(f[i], out[i], f32);
    return r;
}

/* marker equal to f on the border pixels B of the image and `fill` inside */
static double *ora_border_marker(const double *f, long H, long W, double fill)
{
    double *mk = (double *)malloc((size_t)(H * W) * sizeof(double));
    if (!mk) return NULL;
    for (long y = 0; y < H; ++y)
        for (long x = 0; x < W; ++x)
            mk[y * W + x] = (y == 0 || x == 0 || y == H - 1 || x == W - 1) ? f[y * W + x] : fill;
    return mk;
}

/* HFILL(f) = erosion by reconstruction of m_HFILL under f, m_HFILL = f on
 * the border and max f inside (Eq. 8-9). */
long oracle_hfill(const double *f, double *out, long H, long W, int conn)
{
    long n = H * W;
    if (n == 0) return 0;
    double mx = f[0];
    for (long i = 1; i < n; ++i) if (f[i] > mx) mx = f[i];
    double *mk = ora_border_marker(f, H, W, mx);
    if (!mk) return -2;
    long r = oracle_reconstruct(mk, f, out, H, W, conn, ORA_ERODE, n + 1);
    free(mk);
    return r;
}

/* RAOBJ(f) = f - dilation by reconstruction of m_RAOBJ under f, m_RAOBJ = f
 * on the border and min f inside (Eq. 10-11). */
long oracle_raobj(const double *f, double *out, long H, long W, int conn, int f32)
{
    long n = H * W;
    if (n == 0) return 0;
    double mn = f[0];
    for (long i = 1; i < n; ++i) if (f[i] < mn) mn = f[i];
    double *mk = ora_border_marker(f, H, W, mn);
    if (!mk) return -2;
    long r = oracle_reconstruct(mk, f, out, H, W, conn, ORA_DILATE, n + 1);
    for (long i = 0; i < n; ++i) out[i] = ora_sub(f[i], out[i], f32);
    free(mk);
    return r;
}

/* Opening by reconstruction gamma_rec^s(f) = dilation by reconstruction of
 * eps_s(f) under f (Eq. 12). */
long oracle_open_rec(const double *f, double *out, long H, long W, int conn, long s)
{
    long n = H * W;
    if (n == 0) return 0;
    double *mk = (double *)malloc((size_t)n * sizeof(double));
    if (!mk) return -2;
    if (oracle_window(f, mk, H, W, s, ORA_ERODE) != 0) { free(mk); return -2; }
    long r = oracle_reconstruct(mk, f, out, H, W, conn, ORA_DILATE, n + 1);
    free(mk);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Quasi-distance transform (Section 2, Eq. 13-15; Section 3.8, Algorithm 6) */
/* ------------------------------------------------------------------------ */

/* First part, d(f) of Eq. 13 as Algorithm 6 builds it: erode f over and over
 * with eps_1; after the j-th erosion (j = 1, 2, ...) the residual
 * eps_{j-1}(f) - eps_j(f) of each pixel is compared with the largest residual
 * r kept so far and, where it is strictly larger, it replaces r and j
 * replaces d. r and d start at 0: a pixel whose value never drops keeps
 * d = 0, and a residual equal to an earlier one keeps the earlier j.
 * `steps` erosions are applied; once eps_j(f) is constant (j >= max(H, W) - 1
 * for the square, H + W - 2 for the cross) every later residual is 0. */
int oracle_qdt_residual(const double *f, double *r, double *d, long H, long W, int conn, long steps)
{
    long n = H * W;
    if (n == 0) return 0;
    double *cur = (double *)malloc((size_t)n * sizeof(double));
    double *nxt = (double *)malloc((size_t)n * sizeof(double));
    if (!cur || !nxt) { free(cur); free(nxt); return -1; }
    memcpy(cur, f, (size_t)n * sizeof(double));
    for (long i = 0; i < n; ++i) { r[i] = 0.0; d[i] = 0.0; }
    for (long j = 1; j <= steps; ++j) {
        oracle_step(cur, NULL, nxt, H, W, conn, ORA_ERODE);
        for (long i = 0; i < n; ++i) {
            double res = cur[i] - nxt[i];
            if (res > r[i]) { r[i] = res; d[i] = (double)j; }
        }
        double *t = cur; cur = nxt; nxt = t;
    }
    free(cur);
    free(nxt);
    return 0;
}

/* Second part: eta of Eq. 14, applied until a step changes nothing (the
 * limit of Eq. 15). eta(g)(p) = eps_1(g)(p) + 1 where g(p) - eps_1(g)(p) > 1
 * and g(p) elsewhere; each step computes every pixel from the whole previous
 * image. Returns the number of steps that changed something, -1 if max_steps
 * steps all did, -2 on allocation failure. */
long oracle_qdt_lipschitz(const double *g, double *out, long H, long W, int conn, long max_steps)
{
    long n = H * W;
    if (n == 0) return 0;
    double *eps = (double *)malloc((size_t)n * sizeof(double));
    double *tmp = (double *)malloc((size_t)n * sizeof(double));
    if (!eps || !tmp) { free(eps); free(tmp); return -2; }
    memcpy(out, g, (size_t)n * sizeof(double));
    long changing = 0;
    for (;;) {
        if (changing >= max_steps) { changing = -1; break; }
        oracle_step(out, NULL, eps, H, W, conn, ORA_ERODE);
        int changed = 0;
        for (long i = 0; i < n; ++i) {
            tmp[i] = (out[i] - eps[i] > 1.0) ? eps[i] + 1.0 : out[i];
            if (tmp[i] != out[i]) changed = 1;
        }
        if (!changed) break;
        memcpy(out, tmp, (size_t)n * sizeof(double));
        ++changing;
    }
    free(eps);
    free(tmp);
    return changing;
}

/* ------------------------------------------------------------------------ */
/* Granulometry and alternating sequential filters (Section 2, Eq. 16-20)    */
/* ------------------------------------------------------------------------ */

/* gamma_s(f) = delta_s(eps_s(f)) (Eq. 16): s elementary erosions eps_1, then s
 * elementary dilations delta_1 (3x3 square, clipped). phi_s(f) =
 * eps_s(delta_s(f)) (Eq. 19): the same in the other order. first_op is the
 * operation applied first (ORA_ERODE for the opening). */
static int ora_open_close(const double *f, double *out, long H, long W, long s, int first_op)
{
    long n = H * W;
    double *tmp = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!tmp) return -1;
    int second_op = first_op == ORA_ERODE ? ORA_DILATE : ORA_ERODE;
    int rc = oracle_chain(f, NULL, tmp, H, W, 8, first_op, s);
    if (rc == 0) rc = oracle_chain(tmp, NULL, out, H, W, 8, second_op, s);
    free(tmp);
    return rc;
}

int oracle_opening(const double *f, double *out, long H, long W, long s)
{
    return ora_open_close(f, out, H, W, s, ORA_ERODE);
}

int oracle_closing(const double *f, double *out, long H, long W, long s)
{
    return ora_open_close(f, out, H, W, s, ORA_DILATE);
}

/* Granulometric function G_s(f) = sum over P of gamma_s(f) (Eq. 17) for
 * s = 0..smax into G[0..smax] (gamma_0 is f itself), each opening computed
 * from f, and the pixel sum taken row by row in double. The pattern spectrum
 * PS_s = G_s - G_{s+1} (Eq. 18) follows from G. */
int oracle_granulometry(const double *f, long H, long W, long smax, double *G)
{
    long n = H * W;
    double *g = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!g) return -1;
    for (long s = 0; s <= smax; ++s) {
        if (ora_open_close(f, g, H, W, s, ORA_ERODE) != 0) { free(g); return -1; }
        double sum = 0.0;
        for (long i = 0; i < n; ++i) sum += g[i];
        G[s] = sum;
    }
    free(g);
    return 0;
}

/* ASF_s(f) = phi_s(gamma_s(... phi_1(gamma_1(f)))) (Eq. 20): for k = 1..s,
 * the opening gamma_k and then the closing phi_k. */
int oracle_asf(const double *f, double *out, long H, long W, long s)
{
    long n = H * W;
    double *tmp = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!tmp) return -1;
    memcpy(out, f, (size_t)n * sizeof(double));
    for (long k = 1; k <= s; ++k) {
        if (ora_open_close(out, tmp, H, W, k, ORA_ERODE) != 0) { free(tmp); return -1; }
        if (ora_open_close(tmp, out, H, W, k, ORA_DILATE) != 0) { free(tmp); return -1; }
    }
    free(tmp);
    return 0;
}

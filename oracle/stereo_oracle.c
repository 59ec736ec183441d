/*
 * stereo_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow FP64 CPU oracle for the dense road-stereo part of Fan et al.,
 * "Real-Time Dense Stereo Embedded in A UAV for Road Inspection": the perspective
 * warp (§3.1), the matching cost (eq. c), the bilateral aggregation (eq. omega_s,
 * eq. fbs), winner-take-all and the parabola sub-pixel step (§3.2.2, eq. subpixel).
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg load it.
 * It shares no code with the GPU library: it includes none of its headers and the
 * library never links or calls anything here.
 *
 * Every quantity is computed from its definition, with plain loops and no running
 * sums.  Readings taken where the paper is silent:
 *   - warp: a fractional row shift is rounded to the nearest integer,
 *     s_i = floor(s + 0.5); a source column outside the row clamps to the edge;
 *   - eq. (c): mean and standard deviation are population statistics (1/n) over the
 *     w x w block; every image read clamps to the edge in u and v; when
 *     sigma_ref * sigma_tar == 0 the cost is 1 (NCC taken as 0);
 *   - eq. (omega_s), eq. (fbs): sigma0 and sigma1 are used exactly as printed (no
 *     factor 2), the guide image is the reference, and neighbours outside the image
 *     are left out of both sums;
 *   - WTA: the lowest d wins a tie; eq. (subpixel) is applied to the aggregated cost
 *     E; delta = 0 when d* is 0 or D-1 or when the denominator is not positive;
 *   - the target view (the second cost volume of §3.2.1) matches the target block around
 *     x against the reference block around x + [d, 0] with eq. (c), and its aggregation
 *     takes the target image as the guide of eq. (omega_s);
 *   - eq. (lrc) compares the integer WTA disparities of the two views before the
 *     sub-pixel step, in the warped target's columns (the row shift is added to both
 *     disparities and cancels); a partner column outside the image fails the check.
 * Layouts: images are row-major uint8 with a row pitch in bytes; cost and
 * aggregated volumes are double [H][W][D]; disparity maps are double [H][W].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* §3.1: the integer shift applied to a row (round to nearest, halves up). */
int oracle_round_shift(double s) { return (int)floor(s + 0.5); }

/* §3.1: shift every point of target row v to the right by s(v):
 * out(u, v) = tgt(clamp(u - s_i(v)), v). */
void oracle_warp(int W, int H, int pitch, const uint8_t *tgt, const float *shift,
                 uint8_t *out, int out_pitch)
{
    for (int v = 0; v < H; ++v) {
        int si = oracle_round_shift((double)shift[v]);
        for (int u = 0; u < W; ++u)
            out[(size_t)v * out_pitch + u] = tgt[(size_t)v * pitch + clampi(u - si, 0, W - 1)];
    }
}

/* eq. (c): cost of matching reference pixel p = (u, v) at disparity d, i.e. the
 * w x w reference block around p against the target block around p - [d, 0]. */
double oracle_cost(const uint8_t *ref, const uint8_t *tgt, int W, int H, int pitch,
                   int u, int v, int d, int rw)
{
    const int w = 2 * rw + 1;
    const double n = (double)(w * w);
    double sum_r = 0.0, sum_t = 0.0;
    for (int dy = -rw; dy <= rw; ++dy) {
        int y = clampi(v + dy, 0, H - 1);
        for (int dx = -rw; dx <= rw; ++dx) {
            sum_r += ref[(size_t)y * pitch + clampi(u + dx, 0, W - 1)];
            sum_t += tgt[(size_t)y * pitch + clampi(u + dx - d, 0, W - 1)];
        }
    }
    const double mu_r = sum_r / n, mu_t = sum_t / n;
    double var_r = 0.0, var_t = 0.0, cross = 0.0;
    for (int dy = -rw; dy <= rw; ++dy) {
        int y = clampi(v + dy, 0, H - 1);
        for (int dx = -rw; dx <= rw; ++dx) {
            double a = ref[(size_t)y * pitch + clampi(u + dx, 0, W - 1)];
            double b = tgt[(size_t)y * pitch + clampi(u + dx - d, 0, W - 1)];
            var_r += (a - mu_r) * (a - mu_r);
            var_t += (b - mu_t) * (b - mu_t);
            cross += a * b;   /* sum over N+_p of i_ref(q) i_tar(q - [d,0]) */
        }
    }
    const double sig_r = sqrt(var_r / n), sig_t = sqrt(var_t / n);
    const double ss = sig_r * sig_t;
    if (ss == 0.0) return 1.0;
    return (ss + mu_r * mu_t) / ss - cross / (n * ss);
}

/* eq. (c) for every pixel and d in [0, D) of rows [v0, v1): c[(v - v0)][u][d]. */
void oracle_cost_rows(const uint8_t *ref, const uint8_t *tgt, int W, int H, int pitch,
                      int D, int rw, int v0, int v1, double *c)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int v = v0; v < v1; ++v)
        for (int u = 0; u < W; ++u)
            for (int d = 0; d < D; ++d)
                c[((size_t)(v - v0) * W + u) * D + d] = oracle_cost(ref, tgt, W, H, pitch, u, v, d, rw);
}

void oracle_cost_volume(const uint8_t *ref, const uint8_t *tgt, int W, int H, int pitch,
                        int D, int rw, double *c)
{
    oracle_cost_rows(ref, tgt, W, H, pitch, D, rw, 0, H, c);
}

/* eq. (omega_s): bilateral weight between p and its neighbour q (guide: reference). */
double oracle_weight(const uint8_t *ref, int pitch, int up, int vp, int uq, int vq,
                     double sigma0, double sigma1)
{
    double du = (double)(up - uq), dv = (double)(vp - vq);
    double di = (double)ref[(size_t)vp * pitch + up] - (double)ref[(size_t)vq * pitch + uq];
    return exp(-(du * du + dv * dv) / (sigma0 * sigma0) - (di * di) / (sigma1 * sigma1));
}

/* eq. (fbs) for the pixels of rows [v0, v1), reading costs c of rows [cv0, cv1)
 * (layout [(v - cv0)][u][d]); E[(v - v0)][u][d]; wsum[(v - v0)][u] if not NULL. */
void oracle_aggregate_rows(const uint8_t *ref, int W, int H, int pitch, int D, int rb,
                           double sigma0, double sigma1, const double *c, int cv0, int cv1,
                           int v0, int v1, double *E, double *wsum)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int v = v0; v < v1; ++v) {
        for (int u = 0; u < W; ++u) {
            double *e = E + ((size_t)(v - v0) * W + u) * D;
            for (int d = 0; d < D; ++d) e[d] = 0.0;
            double ws = 0.0;
            for (int dy = -rb; dy <= rb; ++dy) {
                int vq = v + dy;
                if (vq < 0 || vq >= H || vq < cv0 || vq >= cv1) continue;
                for (int dx = -rb; dx <= rb; ++dx) {
                    int uq = u + dx;
                    if (uq < 0 || uq >= W) continue;
                    double w = oracle_weight(ref, pitch, u, v, uq, vq, sigma0, sigma1);
                    const double *cq = c + ((size_t)(vq - cv0) * W + uq) * D;
                    ws += w;
                    for (int d = 0; d < D; ++d) e[d] += w * cq[d];
                }
            }
            for (int d = 0; d < D; ++d) e[d] /= ws;
            if (wsum) wsum[(size_t)(v - v0) * W + u] = ws;
        }
    }
}

void oracle_aggregate(const uint8_t *ref, int W, int H, int pitch, int D, int rb,
                      double sigma0, double sigma1, const double *c, double *E, double *wsum)
{
    oracle_aggregate_rows(ref, W, H, pitch, D, rb, sigma0, sigma1, c, 0, H, 0, H, E, wsum);
}

/* §3.2.2: WTA over d, add back the row shift, eq. (subpixel) on E.
 * E holds rows [v0, v1) as [(v - v0)][u][d]; outputs are written for those rows. */
void oracle_wta_rows(int W, int D, const double *E, const float *shift, int v0, int v1,
                     double *disp, int32_t *dstar, double *ebest, double *esecond)
{
    #pragma omp parallel for schedule(static)
    for (int v = v0; v < v1; ++v) {
        int si = oracle_round_shift((double)shift[v]);
        for (int u = 0; u < W; ++u) {
            size_t p = (size_t)(v - v0) * W + u;
            const double *e = E + p * D;
            int b = 0;
            for (int d = 1; d < D; ++d)
                if (e[d] < e[b]) b = d;
            double second = INFINITY;
            for (int d = 0; d < D; ++d)
                if (d != b && e[d] < second) second = e[d];
            double delta = 0.0;
            if (b > 0 && b < D - 1) {
                double den = 2.0 * e[b - 1] + 2.0 * e[b + 1] - 4.0 * e[b];
                if (den > 0.0) delta = (e[b - 1] - e[b + 1]) / den;
            }
            if (disp) disp[p] = (double)b + delta + (double)si;
            if (dstar) dstar[p] = b;
            if (ebest) ebest[p] = e[b];
            if (esecond) esecond[p] = second;
        }
    }
}

/* The whole stereo step for rows [v0, v1) of a pair whose target is already warped:
 * costs of rows [v0 - rb, v1 + rb) (clipped), aggregation, WTA and sub-pixel.
 * Outputs are indexed [(v - v0)][u].  Returns 0, or -1 when out of memory. */
int oracle_stereo_rows(const uint8_t *ref, const uint8_t *tgtw, const float *shift,
                       int W, int H, int pitch, int D, int rw, int rb,
                       double sigma0, double sigma1, int v0, int v1,
                       double *disp, int32_t *dstar, double *ebest, double *esecond)
{
    int cv0 = v0 - rb < 0 ? 0 : v0 - rb;
    int cv1 = v1 + rb > H ? H : v1 + rb;
    double *c = (double *)malloc(sizeof(double) * (size_t)(cv1 - cv0) * W * D);
    double *E = (double *)malloc(sizeof(double) * (size_t)(v1 - v0) * W * D);
    if (!c || !E) { free(c); free(E); return -1; }
    oracle_cost_rows(ref, tgtw, W, H, pitch, D, rw, cv0, cv1, c);
    oracle_aggregate_rows(ref, W, H, pitch, D, rb, sigma0, sigma1, c, cv0, cv1, v0, v1, E, NULL);
    oracle_wta_rows(W, D, E, shift, v0, v1, disp, dstar, ebest, esecond);
    free(c);
    free(E);
    return 0;
}

/* Geometric validity: pixel (u, v) is valid when no read behind its disparity
 * (any d in [0, D), NCC and bilateral windows, m = rw + rb) is clamped, either in
 * the reference, in the warped target, or in the original target behind the warp. */
void oracle_valid_mask(int W, int H, int D, int rw, int rb, const float *shift, uint8_t *mask)
{
    const int m = rw + rb;
    for (int v = 0; v < H; ++v) {
        int s_hi = -(1 << 30), s_lo = 1 << 30;
        for (int y = v - m; y <= v + m; ++y) {
            if (y < 0 || y >= H) continue;
            int si = oracle_round_shift((double)shift[y]);
            if (si > s_hi) s_hi = si;
            if (si < s_lo) s_lo = si;
        }
        int ulo = m + D - 1 + (s_hi > 0 ? s_hi : 0);
        int uhi = W - 1 - m + (s_lo < 0 ? s_lo : 0);
        for (int u = 0; u < W; ++u) {
            int ok = v >= m && v <= H - 1 - m && u >= ulo && u <= uhi;
            mask[(size_t)v * W + u] = (uint8_t)ok;
        }
    }
}

/* The target view: the cost of target pixel x = (u, v) at disparity d, i.e. eq. (c) with the
 * target block around x and the reference block around x + [d, 0] -- eq. (c) with the roles of
 * the two images exchanged and the disparity negated. */
double oracle_cost_tar(const uint8_t *ref, const uint8_t *tgtw, int W, int H, int pitch,
                       int u, int v, int d, int rw)
{
    return oracle_cost(tgtw, ref, W, H, pitch, u, v, -d, rw);
}

/* Target-view WTA for rows [v0, v1): target-view costs of rows [v0 - rb, v1 + rb), eq. (fbs)
 * with the warped target as the guide, lowest d on ties.  dstar / ebest / esecond are
 * indexed [(v - v0)][u] (u a column of the warped target).  Returns 0, or -1 when out of
 * memory. */
int oracle_target_view_rows(const uint8_t *ref, const uint8_t *tgtw, int W, int H, int pitch,
                            int D, int rw, int rb, double sigma0, double sigma1, int v0, int v1,
                            int32_t *dstar, double *ebest, double *esecond)
{
    int cv0 = v0 - rb < 0 ? 0 : v0 - rb;
    int cv1 = v1 + rb > H ? H : v1 + rb;
    double *c = (double *)malloc(sizeof(double) * (size_t)(cv1 - cv0) * W * D);
    double *E = (double *)malloc(sizeof(double) * (size_t)(v1 - v0) * W * D);
    float *zero = (float *)calloc((size_t)H, sizeof(float));
    if (!c || !E || !zero) { free(c); free(E); free(zero); return -1; }
    #pragma omp parallel for schedule(dynamic, 1)
    for (int v = cv0; v < cv1; ++v)
        for (int u = 0; u < W; ++u)
            for (int d = 0; d < D; ++d)
                c[((size_t)(v - cv0) * W + u) * D + d] = oracle_cost_tar(ref, tgtw, W, H, pitch, u, v, d, rw);
    oracle_aggregate_rows(tgtw, W, H, pitch, D, rb, sigma0, sigma1, c, cv0, cv1, v0, v1, E, NULL);
    oracle_wta_rows(W, D, E, zero, v0, v1, NULL, dstar, ebest, esecond);
    free(c);
    free(E);
    free(zero);
    return 0;
}

/* eq. (lrc): reference pixel (u, v) keeps its disparity when
 * (d_ref(u, v) - d_tar(u - d_ref(u, v), v))^2 <= delta_r; both maps are integer WTA disparities
 * [H][W] of the warped pair, and a partner column u - d_ref < 0 fails. */
void oracle_lr_check(int W, int H, const int32_t *dref, const int32_t *dtar, double delta_r, uint8_t *ok)
{
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            int dr = dref[(size_t)v * W + u], x = u - dr;
            int pass = 0;
            if (x >= 0 && x < W) {
                double diff = (double)(dr - dtar[(size_t)v * W + x]);
                pass = diff * diff <= delta_r;
            }
            ok[(size_t)v * W + u] = (uint8_t)pass;
        }
}

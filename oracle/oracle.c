/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the receive beamformer of
 * SUPRA (Goebl, Navab, Hennersperger, "SUPRA: Open Source Software Defined
 * Ultrasound Processing for Real-Time Applications", arXiv:1711.06127).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py load this library.  It shares no source,
 * header, table or helper with the CUDA path, and nothing here is reachable
 * from the product library.
 *
 * The paper names the steps of the pipeline (Sec. 1, step list "receive
 * beamforming", Sec. 2 method list items 1-2: dynamic receive beamforming for
 * a flexible scanline layout and multi-line acquisitions, delay-and-sum of raw
 * channel data after A/D conversion, citing Shattuck et al. 1984) but prints no
 * formula.  What follows is the textbook delay-and-sum written out directly:
 *
 *   For scanline l (origin o_l, unit direction d_l, transmit event t = line_tx[l]
 *   with transmit origin o_t) and depth r_i = depth0 + i*depth_step, the image
 *   point is p = o_l + r_i d_l.  Element e at x_e receives the echo of p after
 *       tau_e = (|p - o_t| + |p - x_e|) / c - t0          (two-way path)
 *   which is channel sample s = tau_e * fs, read by linear interpolation
 *   between floor(s) and floor(s)+1 (samples outside [0, n_s-1] read as 0).
 *   Dynamic aperture (F-number): centre q = (p_x, p_y) clamped to the array's
 *   extent, half width a = max(p_z / (2F), min_half_aperture); e is active iff
 *   |x_e - q| <= a on each lateral axis.  Apodization is the product over the
 *   two lateral axes of the window evaluated at u = (x_e - q)/a.
 *       RF(l, i) = sum_active w_e v_e / sum_active w_e      (0 if sum w = 0)
 *
 * Readings taken where the paper is silent: spherical transmit delay from the
 * transmit origin, normalisation by the weight sum, linear interpolation, a
 * separable square aperture, zero padding outside the record.
 *
 * Plane-wave transmits (planned in the paper's outlook, Sec. 2, citing
 * ultrafast plane-wave imaging): a transmit t with a nonzero direction n_t
 * is a plane wave that passes its origin o_t at time 0, so it reaches p after
 * n_t.(p - o_t) / c (n_t normalised) instead of |p - o_t| / c.  Coherent
 * compounding: each line is reconstructed from every transmit event of the
 * frame and the per-transmit delay-and-sum values are averaged,
 *     RF_comp(l, i) = (1 / n_tx) sum_t RF_t(l, i).
 *
 * The minimum-variance (Capon) beamformer below is not in the paper; it is the
 * textbook spatially smoothed MV estimator with diagonal loading.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_WINDOW_RECT 0
#define OR_WINDOW_HANN 1
#define OR_WINDOW_HAMMING 2

typedef struct {
    int32_t n_el;
    const double *elem;        /* [n_el][3] element positions, metres         */
    int32_t n_tx;
    const double *tx_origin;   /* [n_tx][3]                                   */
    int32_t n_lines;
    const double *line_origin; /* [n_lines][3]                                */
    const double *line_dir;    /* [n_lines][3], unit vectors                  */
    const int32_t *line_tx;    /* [n_lines] transmit event of each line       */
    int32_t n_depth;
    double depth0, depth_step; /* r_i = depth0 + i * depth_step               */
    double c, fs, t0;          /* speed of sound, sampling rate, record start */
    double fnumber, min_half_aperture;
    int32_t window;            /* OR_WINDOW_*                                 */
    int32_t n_s;               /* samples per channel                         */
    const double *tx_dir;      /* NULL or [n_tx][3]: nonzero = plane wave     */
    int32_t compound;          /* 1: every line averages all transmits        */
} or_geom;

static double dist3(const double *a, const double *b)
{
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* apodization window on u in [-1, 1] (u = 0 at the aperture centre) */
static double window_at(int window, double u)
{
    const double pi = 3.14159265358979323846;
    if (window == OR_WINDOW_HANN) return 0.5 * (1.0 + cos(pi * u));
    if (window == OR_WINDOW_HAMMING) return 0.54 + 0.46 * cos(pi * u);
    return 1.0;
}

/* channel sample j of one element's record; zero outside the record */
static double sample_at(const int16_t *rec, int32_t n_s, long j)
{
    if (j < 0 || j >= n_s) return 0.0;
    return (double)rec[j];
}

static void array_extent(const or_geom *g, double ext[4])
{
    ext[0] = ext[2] = INFINITY;
    ext[1] = ext[3] = -INFINITY;
    for (int e = 0; e < g->n_el; ++e) {
        const double *x = g->elem + 3 * e;
        if (x[0] < ext[0]) ext[0] = x[0];
        if (x[0] > ext[1]) ext[1] = x[0];
        if (x[1] < ext[2]) ext[2] = x[1];
        if (x[1] > ext[3]) ext[3] = x[1];
    }
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/*
 * The image point, aperture centre and aperture half width of (line, i).
 */
static void point_and_aperture(const or_geom *g, const double ext[4], int32_t line, int32_t i,
                               double p[3], double q[2], double *a)
{
    const double *o = g->line_origin + 3 * line;
    const double *d = g->line_dir + 3 * line;
    double r = g->depth0 + (double)i * g->depth_step;
    for (int k = 0; k < 3; ++k) p[k] = o[k] + r * d[k];
    q[0] = clampd(p[0], ext[0], ext[1]);
    q[1] = clampd(p[1], ext[2], ext[3]);
    double a_f = p[2] / (2.0 * g->fnumber);
    *a = a_f > g->min_half_aperture ? a_f : g->min_half_aperture;
}

/* Transmit path of event t to point p: |p - o_t| (spherical), or
 * n_t . (p - o_t) for a plane wave of direction n_t. */
static double tx_path_to(const or_geom *g, int32_t t, const double p[3])
{
    const double *o_t = g->tx_origin + 3 * t;
    if (g->tx_dir) {
        const double *n = g->tx_dir + 3 * t;
        double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (len > 0.0)
            return (n[0] * (p[0] - o_t[0]) + n[1] * (p[1] - o_t[1]) + n[2] * (p[2] - o_t[2])) / len;
    }
    return dist3(p, o_t);
}

/* delay-and-sum value at (line, depth index i) from transmit event t; ch_tx =
 * records of that transmit event, [n_el][n_s] */
static double das_point_tx(const or_geom *g, const double ext[4], const int16_t *ch_tx, int32_t t,
                           int32_t line, int32_t i)
{
    double p[3], q[2], a;
    point_and_aperture(g, ext, line, i, p, q, &a);
    double tx_path = tx_path_to(g, t, p);
    double num = 0.0, den = 0.0;
    for (int e = 0; e < g->n_el; ++e) {
        const double *x = g->elem + 3 * e;
        double ux = (x[0] - q[0]) / a, uy = (x[1] - q[1]) / a;
        if (fabs(ux) > 1.0 || fabs(uy) > 1.0) continue;     /* outside the aperture */
        double w = window_at(g->window, ux) * window_at(g->window, uy);
        double tau = (tx_path + dist3(p, x)) / g->c - g->t0;
        double s = tau * g->fs;
        double k = floor(s);
        double phi = s - k;
        const int16_t *rec = ch_tx + (long)e * g->n_s;
        double v = (1.0 - phi) * sample_at(rec, g->n_s, (long)k) + phi * sample_at(rec, g->n_s, (long)k + 1);
        num += w * v;
        den += w;
    }
    return den > 0.0 ? num / den : 0.0;
}

/* delay-and-sum value at (line, i) from the line's own transmit event */
static double das_point(const or_geom *g, const double ext[4], const int16_t *ch_tx, int32_t line, int32_t i)
{
    return das_point_tx(g, ext, ch_tx, g->line_tx[line], line, i);
}

/* Whole frame: ch [n_tx][n_el][n_s] -> rf [n_lines][n_depth]; with compounding
 * every line averages the delay-and-sum values of all transmit events. */
void oracle_das(const or_geom *g, const int16_t *ch, double *rf)
{
    double ext[4];
    array_extent(g, ext);
    long rec_tx = (long)g->n_el * g->n_s;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t l = 0; l < g->n_lines; ++l) {
        for (int32_t i = 0; i < g->n_depth; ++i) {
            double v;
            if (g->compound) {
                v = 0.0;
                for (int32_t t = 0; t < g->n_tx; ++t) v += das_point_tx(g, ext, ch + rec_tx * t, t, l, i);
                v /= (double)g->n_tx;
            } else {
                v = das_point(g, ext, ch + rec_tx * g->line_tx[l], l, i);
            }
            rf[(long)l * g->n_depth + i] = v;
        }
    }
}

/*
 * The same delay-and-sum loops in single precision, for a CPU timing column
 * beside the FP64 oracle (the two differ only in the precision of the
 * arithmetic).  It is a timing reference, not an oracle: tests compare it with
 * oracle_das within single-precision rounding.
 */
static float window_at_f(int window, float u)
{
    const float pi = 3.14159265358979f;
    if (window == OR_WINDOW_HANN) return 0.5f * (1.0f + cosf(pi * u));
    if (window == OR_WINDOW_HAMMING) return 0.54f + 0.46f * cosf(pi * u);
    return 1.0f;
}

static float das_point_tx_f(const or_geom *g, const float *elem, const float ext[4], const int16_t *ch_tx,
                            int32_t t, int32_t line, int32_t i)
{
    const double *od = g->line_origin + 3 * line, *dd = g->line_dir + 3 * line;
    const float r = (float)g->depth0 + (float)i * (float)g->depth_step;
    float p[3], q[2];
    for (int k = 0; k < 3; ++k) p[k] = (float)od[k] + r * (float)dd[k];
    q[0] = p[0] < ext[0] ? ext[0] : (p[0] > ext[1] ? ext[1] : p[0]);
    q[1] = p[1] < ext[2] ? ext[2] : (p[1] > ext[3] ? ext[3] : p[1]);
    float a = p[2] / (2.0f * (float)g->fnumber);
    if (a < (float)g->min_half_aperture) a = (float)g->min_half_aperture;
    const double *ot = g->tx_origin + 3 * t;
    float tx_path;
    if (g->tx_dir && (g->tx_dir[3 * t] != 0.0 || g->tx_dir[3 * t + 1] != 0.0 || g->tx_dir[3 * t + 2] != 0.0)) {
        const double *n = g->tx_dir + 3 * t;
        const float len = sqrtf((float)(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]));
        tx_path = ((float)n[0] * (p[0] - (float)ot[0]) + (float)n[1] * (p[1] - (float)ot[1]) +
                   (float)n[2] * (p[2] - (float)ot[2])) / len;
    } else {
        const float dx = p[0] - (float)ot[0], dy = p[1] - (float)ot[1], dz = p[2] - (float)ot[2];
        tx_path = sqrtf(dx * dx + dy * dy + dz * dz);
    }
    const float inv_c = 1.0f / (float)g->c, fs = (float)g->fs, t0 = (float)g->t0;
    float num = 0.0f, den = 0.0f;
    for (int e = 0; e < g->n_el; ++e) {
        const float *x = elem + 3 * e;
        const float ux = (x[0] - q[0]) / a, uy = (x[1] - q[1]) / a;
        if (fabsf(ux) > 1.0f || fabsf(uy) > 1.0f) continue;
        const float w = window_at_f(g->window, ux) * window_at_f(g->window, uy);
        const float dx = p[0] - x[0], dy = p[1] - x[1], dz = p[2] - x[2];
        const float s = ((tx_path + sqrtf(dx * dx + dy * dy + dz * dz)) * inv_c - t0) * fs;
        const float k = floorf(s);
        const float phi = s - k;
        const long j = (long)k;
        const int16_t *rec = ch_tx + (long)e * g->n_s;
        const float v0 = (j >= 0 && j < g->n_s) ? (float)rec[j] : 0.0f;
        const float v1 = (j + 1 >= 0 && j + 1 < g->n_s) ? (float)rec[j + 1] : 0.0f;
        num += w * ((1.0f - phi) * v0 + phi * v1);
        den += w;
    }
    return den > 0.0f ? num / den : 0.0f;
}

void oracle_das_f32(const or_geom *g, const int16_t *ch, float *rf)
{
    double extd[4];
    array_extent(g, extd);
    const float ext[4] = {(float)extd[0], (float)extd[1], (float)extd[2], (float)extd[3]};
    float *elem = (float *)malloc(sizeof(float) * 3 * (size_t)(g->n_el > 0 ? g->n_el : 1));
    if (!elem) return;
    for (int k = 0; k < 3 * g->n_el; ++k) elem[k] = (float)g->elem[k];
    long rec_tx = (long)g->n_el * g->n_s;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t l = 0; l < g->n_lines; ++l) {
        for (int32_t i = 0; i < g->n_depth; ++i) {
            float v;
            if (g->compound) {
                v = 0.0f;
                for (int32_t t = 0; t < g->n_tx; ++t) v += das_point_tx_f(g, elem, ext, ch + rec_tx * t, t, l, i);
                v /= (float)g->n_tx;
            } else {
                v = das_point_tx_f(g, elem, ext, ch + rec_tx * g->line_tx[l], g->line_tx[l], l, i);
            }
            rf[(long)l * g->n_depth + i] = v;
        }
    }
    free(elem);
}

/* Selected points only: point k is (lines[k], depths[k]); its transmit
 * event's records are at ch_tx[k] ([n_el][n_s]).  Used for sampled checks of
 * frames too large for a full CPU pass (one transmit per line: no
 * compounding). */
void oracle_das_points(const or_geom *g, int32_t n_pts, const int32_t *lines, const int32_t *depths,
                       const int16_t *const *ch_tx, double *out)
{
    double ext[4];
    array_extent(g, ext);
#pragma omp parallel for schedule(dynamic, 64)
    for (int32_t k = 0; k < n_pts; ++k)
        out[k] = das_point(g, ext, ch_tx[k], lines[k], depths[k]);
}

/* The aperture of (line, i): active-element mask and weights (diagnostics for
 * tests: weight sums, element counts, distance of each element to the aperture
 * edge).  mask[e] = 1 if active; w[e] = window weight (0 if inactive);
 * margin[e] = a - max(|x_e - q|) in metres (negative = outside). */
void oracle_aperture(const or_geom *g, int32_t line, int32_t i, int32_t *mask, double *w, double *margin)
{
    double ext[4], p[3], q[2], a;
    array_extent(g, ext);
    point_and_aperture(g, ext, line, i, p, q, &a);
    for (int e = 0; e < g->n_el; ++e) {
        const double *x = g->elem + 3 * e;
        double ux = (x[0] - q[0]) / a, uy = (x[1] - q[1]) / a;
        double m = fabs(x[0] - q[0]) > fabs(x[1] - q[1]) ? fabs(x[0] - q[0]) : fabs(x[1] - q[1]);
        margin[e] = a - m;
        int on = !(fabs(ux) > 1.0 || fabs(uy) > 1.0);
        mask[e] = on;
        w[e] = on ? window_at(g->window, ux) * window_at(g->window, uy) : 0.0;
    }
}

/* Delayed, interpolated samples of the active elements at (line, i), in
 * element order; returns the count.  x[] must hold n_el values.  This is the
 * vector the minimum-variance beamformer and the apodization network consume. */
int32_t oracle_delayed_samples(const or_geom *g, const int16_t *ch_tx, int32_t line, int32_t i, double *x,
                               int32_t *elems)
{
    double ext[4], p[3], q[2], a;
    array_extent(g, ext);
    point_and_aperture(g, ext, line, i, p, q, &a);
    double tx_path = tx_path_to(g, g->line_tx[line], p);
    int32_t m = 0;
    for (int e = 0; e < g->n_el; ++e) {
        const double *xe = g->elem + 3 * e;
        double ux = (xe[0] - q[0]) / a, uy = (xe[1] - q[1]) / a;
        if (fabs(ux) > 1.0 || fabs(uy) > 1.0) continue;
        double s = ((tx_path + dist3(p, xe)) / g->c - g->t0) * g->fs;
        double k = floor(s), phi = s - k;
        const int16_t *rec = ch_tx + (long)e * g->n_s;
        x[m] = (1.0 - phi) * sample_at(rec, g->n_s, (long)k) + phi * sample_at(rec, g->n_s, (long)k + 1);
        if (elems) elems[m] = e;
        ++m;
    }
    return m;
}

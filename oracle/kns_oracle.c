/*
 * kns_oracle.c -- plain, slow FP64 oracle of the KiloNeuS sphere-tracing path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library: it reads the canonical FP32
 * weight array (the layout every caller passes in) and computes everything in
 * double precision with the C library's sin/cos/exp/log1p.
 *
 * What it computes, and where the paper defines it:
 *   - positional encoding gamma_L (Sec. 3.1, Eq. 1), raw coordinates first,
 *     then per frequency k the sines of x,y,z and then the cosines of x,y,z;
 *   - cell map m(x) (Sec. 3.1): floor of the scaled coordinate, clamped to
 *     [0, N-1], cell = ix + N*(iy + N*iz);
 *   - SDF MLP f (Sec. 3.1, Eq. 2): softplus_beta hidden layers, linear output
 *     [d, z]; softplus_beta(s) = max(s,0) + log1p(exp(-beta|s|))/beta;
 *   - analytic input gradient of d by reverse mode through the layers and the
 *     encoding, normal n = grad d / |grad d| (Sec. 3.1);
 *   - colour MLP g (Sec. 3.1, Eq. 3): input [z, n, gamma_Ld(v), x (optional)],
 *     ReLU hidden layers, sigmoid output;
 *   - sphere tracing inside the bounding-box interval (Sec. 3.4.1, after
 *     Hart 1993): test |d| < eps, else t += d, a miss when t leaves the
 *     interval [max(t_near, 0), t_far] or the step budget is spent; normal and
 *     colour at the hit;
 *   - optional occupancy-mask empty-space skipping with an integer 3D-DDA
 *     (Amanatides & Woo 1987) to the entry of the next occupied voxel;
 *   - brute-force root marching (fixed small step + bisection) for pins.
 *
 * Alongside each traced ray it records decision margins: how close each
 * threshold test (|d| vs eps, t vs t_far, floor at a cell or voxel face, DDA
 * axis choice) came to flipping.  A ray whose margins all exceed small bounds
 * takes the same decisions in any accurate FP32 implementation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define KO_MAXW 256
#define KO_MAXIN 256
#define KO_MAXLAYERS 16

typedef struct {
    int32_t N, pe_pos_L, pe_dir_L, sdf_hidden, sdf_width, feat_dim, col_hidden, col_width,
        col_use_x, occ_res;
    double beta;
    double bmin[3], bmax[3];
} ko_desc;

/* ------------------------------------------------------------------ shapes */
static int sdf_in_dim(const ko_desc *g) { return 3 + 6 * g->pe_pos_L; }
static int col_in_dim(const ko_desc *g) {
    return g->feat_dim + 3 + 3 + 6 * g->pe_dir_L + (g->col_use_x ? 3 : 0);
}
static int sdf_dims(const ko_desc *g, int *dims) {
    int n = 0;
    dims[n++] = sdf_in_dim(g);
    for (int i = 0; i < g->sdf_hidden; i++) dims[n++] = g->sdf_width;
    dims[n++] = 1 + g->feat_dim;
    return n; /* number of dims = layers + 1 */
}
static int col_dims(const ko_desc *g, int *dims) {
    int n = 0;
    dims[n++] = col_in_dim(g);
    for (int i = 0; i < g->col_hidden; i++) dims[n++] = g->col_width;
    dims[n++] = 3;
    return n;
}
static int64_t count_params(const int *dims, int nd) {
    int64_t p = 0;
    for (int l = 0; l + 1 < nd; l++) p += (int64_t)dims[l] * dims[l + 1] + dims[l + 1];
    return p;
}
int64_t ko_params_sdf(const ko_desc *g) {
    int d[KO_MAXLAYERS + 2];
    return count_params(d, sdf_dims(g, d));
}
int64_t ko_params_col(const ko_desc *g) {
    int d[KO_MAXLAYERS + 2];
    return count_params(d, col_dims(g, d));
}
int64_t ko_params_cell(const ko_desc *g) { return ko_params_sdf(g) + ko_params_col(g); }

/* ---------------------------------------------------- Eq. 1: encoding */
/* out = [p_0..p_{n-1}, for k: sin(2^k pi p_c) for c, cos(2^k pi p_c) for c] */
void ko_pe(int L, int n, const double *p, double *out) {
    int o = 0;
    for (int c = 0; c < n; c++) out[o++] = p[c];
    for (int k = 0; k < L; k++) {
        double f = ldexp(M_PI, k);
        for (int c = 0; c < n; c++) out[o++] = sin(f * p[c]);
        for (int c = 0; c < n; c++) out[o++] = cos(f * p[c]);
    }
}

/* ------------------------------------------------------------ activations */
double ko_softplus(double s, double beta) { return fmax(s, 0.0) + log1p(exp(-beta * fabs(s))) / beta; }
/* d softplus_beta / ds = sigmoid(beta s) */
static double dsoftplus(double s, double beta) {
    double e = exp(-beta * fabs(s));
    return s >= 0 ? 1.0 / (1.0 + e) : e / (1.0 + e);
}
static double sigmoid(double s) {
    if (s >= 0) return 1.0 / (1.0 + exp(-s));
    double e = exp(s);
    return e / (1.0 + e);
}

/* --------------------------------------------------------- Sec. 3.1: m(x) */
static double cell_scale(const ko_desc *g, int res, int a) { return (double)res / (g->bmax[a] - g->bmin[a]); }

/* index of x along axis a on a res-cell grid, floor then clamp */
static int grid_index(const ko_desc *g, int res, int a, double x) {
    double u = (x - g->bmin[a]) * cell_scale(g, res, a);
    double f = floor(u);
    if (f < 0) f = 0;
    if (f > res - 1) f = res - 1;
    return (int)f;
}

/* distance from x to the nearest interior face (planes 1..res-1) of a res grid */
static double interior_face_distance(const ko_desc *g, int res, const double x[3]) {
    double best = INFINITY;
    for (int a = 0; a < 3; a++) {
        double s = cell_scale(g, res, a);
        double u = (x[a] - g->bmin[a]) * s;
        double j = floor(u + 0.5); /* nearest plane index */
        if (j < 1) j = 1;
        if (j > res - 1) j = res - 1;
        double dist = fabs(u - j) / s;
        if (dist < best) best = dist;
    }
    return best;
}

int ko_cell(const ko_desc *g, const double x[3]) {
    int i0 = grid_index(g, g->N, 0, x[0]);
    int i1 = grid_index(g, g->N, 1, x[1]);
    int i2 = grid_index(g, g->N, 2, x[2]);
    return i0 + g->N * (i1 + g->N * i2);
}

/* ------------------------------------------- Eq. 2: SDF MLP (+ gradient) */
/* Evaluates [d, z] of cell `cell` at x.  feat (feat_dim) and grad (3) may be NULL. */
double ko_sdf_eval(const ko_desc *g, const float *weights, int cell, const double x[3], double *feat,
                   double *grad) {
    int dims[KO_MAXLAYERS + 2];
    int nd = sdf_dims(g, dims);
    int nl = nd - 1;
    const float *w = weights + (int64_t)cell * ko_params_cell(g);
    /* activations: act[l] is the input of layer l; pre[l] the pre-activation of layer l */
    static __thread double act[KO_MAXLAYERS + 1][KO_MAXIN];
    static __thread double pre[KO_MAXLAYERS][KO_MAXW];
    const float *Wl[KO_MAXLAYERS], *bl[KO_MAXLAYERS];
    int64_t off = 0;
    for (int l = 0; l < nl; l++) {
        Wl[l] = w + off;
        bl[l] = w + off + (int64_t)dims[l] * dims[l + 1];
        off += (int64_t)dims[l] * dims[l + 1] + dims[l + 1];
    }
    ko_pe(g->pe_pos_L, 3, x, act[0]);
    for (int l = 0; l < nl; l++) {
        for (int o = 0; o < dims[l + 1]; o++) {
            double s = (double)bl[l][o];
            for (int i = 0; i < dims[l]; i++) s += (double)Wl[l][(int64_t)o * dims[l] + i] * act[l][i];
            pre[l][o] = s;
            act[l + 1][o] = (l + 1 < nl) ? ko_softplus(s, g->beta) : s;
        }
    }
    double d = act[nl][0];
    if (feat)
        for (int k = 0; k < g->feat_dim; k++) feat[k] = act[nl][1 + k];
    if (grad) {
        /* reverse mode: delta = d d / d act[l] */
        double delta[KO_MAXIN], nxt[KO_MAXIN];
        for (int i = 0; i < dims[nl - 1]; i++) delta[i] = (double)Wl[nl - 1][i]; /* row 0 = d */
        for (int l = nl - 2; l >= 0; l--) {
            /* through the softplus of layer l's output, then W_l^T */
            for (int o = 0; o < dims[l + 1]; o++) delta[o] *= dsoftplus(pre[l][o], g->beta);
            for (int i = 0; i < dims[l]; i++) {
                double s = 0;
                for (int o = 0; o < dims[l + 1]; o++) s += (double)Wl[l][(int64_t)o * dims[l] + i] * delta[o];
                nxt[i] = s;
            }
            memcpy(delta, nxt, sizeof(double) * dims[l]);
        }
        /* through the encoding Jacobian: d/dx sin(f x) = f cos(f x), d/dx cos(f x) = -f sin(f x) */
        for (int c = 0; c < 3; c++) {
            double gc = delta[c];
            for (int k = 0; k < g->pe_pos_L; k++) {
                double f = ldexp(M_PI, k);
                gc += delta[3 + 6 * k + c] * f * cos(f * x[c]);
                gc -= delta[3 + 6 * k + 3 + c] * f * sin(f * x[c]);
            }
            grad[c] = gc;
        }
    }
    return d;
}

/* ---------------------------------------------------- Eq. 3: colour MLP */
void ko_colour_eval(const ko_desc *g, const float *weights, int cell, const double x[3], const double *feat,
                    const double n[3], const double v[3], double rgb[3]) {
    int dims[KO_MAXLAYERS + 2];
    int nd = col_dims(g, dims);
    int nl = nd - 1;
    const float *w = weights + (int64_t)cell * ko_params_cell(g) + ko_params_sdf(g);
    double a[KO_MAXIN], b[KO_MAXIN];
    int u = 0;
    for (int k = 0; k < g->feat_dim; k++) a[u++] = feat[k];
    for (int c = 0; c < 3; c++) a[u++] = n[c];
    ko_pe(g->pe_dir_L, 3, v, a + u);
    u += 3 + 6 * g->pe_dir_L;
    if (g->col_use_x)
        for (int c = 0; c < 3; c++) a[u++] = x[c];
    int64_t off = 0;
    for (int l = 0; l < nl; l++) {
        const float *W = w + off, *bias = w + off + (int64_t)dims[l] * dims[l + 1];
        off += (int64_t)dims[l] * dims[l + 1] + dims[l + 1];
        for (int o = 0; o < dims[l + 1]; o++) {
            double s = (double)bias[o];
            for (int i = 0; i < dims[l]; i++) s += (double)W[(int64_t)o * dims[l] + i] * a[i];
            b[o] = (l + 1 < nl) ? fmax(s, 0.0) : sigmoid(s);
        }
        memcpy(a, b, sizeof(double) * dims[l + 1]);
    }
    for (int c = 0; c < 3; c++) rgb[c] = a[c];
}

/* batch: d, z, grad at points, cell by m(x) */
void ko_sdf_batch(const ko_desc *g, const float *weights, int64_t n, const double *pts, double *d, double *feat,
                  double *grad, int32_t *cells) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int c = ko_cell(g, pts + 3 * i);
        if (cells) cells[i] = c;
        d[i] = ko_sdf_eval(g, weights, c, pts + 3 * i, feat ? feat + i * g->feat_dim : NULL,
                           grad ? grad + 3 * i : NULL);
    }
}

/* ------------------------------------------------------------ occupancy */
/* occupied(voxel) <=> |d(voxel centre)| < voxel diagonal; bit = ix + R*(iy + R*iz) */
void ko_occupancy(const ko_desc *g, const float *weights, int res, double thresh, uint64_t *bits) {
    int64_t nvox = (int64_t)res * res * res;
    memset(bits, 0, sizeof(uint64_t) * ((nvox + 63) / 64));
#pragma omp parallel for schedule(static)
    for (int64_t w = 0; w < (nvox + 63) / 64; w++) {
        uint64_t word = 0;
        for (int b = 0; b < 64; b++) {
            int64_t v = w * 64 + b;
            if (v >= nvox) break;
            int ix = (int)(v % res), iy = (int)((v / res) % res), iz = (int)(v / ((int64_t)res * res));
            double x[3] = {g->bmin[0] + (ix + 0.5) * (g->bmax[0] - g->bmin[0]) / res,
                           g->bmin[1] + (iy + 0.5) * (g->bmax[1] - g->bmin[1]) / res,
                           g->bmin[2] + (iz + 0.5) * (g->bmax[2] - g->bmin[2]) / res};
            double d = ko_sdf_eval(g, weights, ko_cell(g, x), x, NULL, NULL);
            if (fabs(d) < thresh) word |= (uint64_t)1 << b;
        }
        bits[w] = word;
    }
}

static int occ_test(const uint64_t *bits, int res, int ix, int iy, int iz) {
    int64_t v = ix + (int64_t)res * (iy + (int64_t)res * iz);
    return (int)((bits[v >> 6] >> (v & 63)) & 1u);
}

/* ----------------------------------------------------------------- rays */
/* camera: c2w[12] row-major 3x4 (columns right, down, forward, position), fx, fy, cx, cy */
void ko_ray(const float *cam, int i, int j, double o[3], double w[3]) {
    double dc[3] = {((double)j + 0.5 - cam[14]) / cam[12], ((double)i + 0.5 - cam[15]) / cam[13], 1.0};
    double nrm = 0;
    for (int r = 0; r < 3; r++) {
        w[r] = cam[4 * r + 0] * dc[0] + cam[4 * r + 1] * dc[1] + cam[4 * r + 2] * dc[2];
        nrm += w[r] * w[r];
        o[r] = cam[4 * r + 3];
    }
    nrm = sqrt(nrm);
    for (int r = 0; r < 3; r++) w[r] /= nrm;
}

/* slab test against the box; returns 1 and [tn, tf] on overlap with t >= 0 */
int ko_clip(const ko_desc *g, const double o[3], const double w[3], double *tn, double *tf, double *margin) {
    double a = -INFINITY, b = INFINITY;
    for (int k = 0; k < 3; k++) {
        if (w[k] != 0.0) {
            double t1 = (g->bmin[k] - o[k]) / w[k], t2 = (g->bmax[k] - o[k]) / w[k];
            double lo = fmin(t1, t2), hi = fmax(t1, t2);
            if (lo > a) a = lo;
            if (hi < b) b = hi;
        } else if (o[k] < g->bmin[k] || o[k] > g->bmax[k]) {
            *margin = fmin(*margin, fmin(fabs(o[k] - g->bmin[k]), fabs(o[k] - g->bmax[k])));
            return 0;
        }
    }
    *margin = fmin(*margin, fmin(fabs(b - a), fabs(b)));
    if (a > b || b < 0) return 0;
    *tn = a > 0 ? a : 0.0;
    *tf = b;
    return 1;
}

/* Integer 3D-DDA from voxel v (containing o + t w) to the entry of the next occupied voxel.
 * Returns 1 with *te and v updated, or 0 if the ray leaves the grid (or passes tf) first. */
static int dda_next(const ko_desc *g, const uint64_t *bits, int res, const double o[3], const double w[3], int v[3],
                    double tf, double *te, double *m_dda, double *m_t) {
    for (;;) {
        double tm[3];
        for (int a = 0; a < 3; a++) {
            if (w[a] == 0.0) {
                tm[a] = INFINITY;
                continue;
            }
            double h = (g->bmax[a] - g->bmin[a]) / res;
            double plane = g->bmin[a] + (double)(v[a] + (w[a] > 0 ? 1 : 0)) * h;
            tm[a] = (plane - o[a]) / w[a];
        }
        int ax = 0;
        if (tm[1] < tm[ax]) ax = 1;
        if (tm[2] < tm[ax]) ax = 2;
        for (int a = 0; a < 3; a++)
            if (a != ax && isfinite(tm[a])) *m_dda = fmin(*m_dda, tm[a] - tm[ax]);
        v[ax] += w[ax] > 0 ? 1 : -1;
        if (v[ax] < 0 || v[ax] >= res) return 0;
        *m_t = fmin(*m_t, fabs(tm[ax] - tf));
        if (tm[ax] > tf) return 0;
        if (occ_test(bits, res, v[0], v[1], v[2])) {
            *te = tm[ax];
            return 1;
        }
    }
}

/* For pins: from x(t) (in an empty voxel), the DDA's entry t and voxel of the next occupied voxel.
 * Returns 1 if found (t_entry, vox[3] set), 0 if the ray leaves the grid first. */
int ko_first_occupied(const ko_desc *g, const uint64_t *bits, const double o[3], const double w[3], double t,
                      double *t_entry, int32_t vox[3]) {
    int res = g->occ_res;
    double tn, tf, m = INFINITY;
    if (!ko_clip(g, o, w, &tn, &tf, &m)) return 0;
    double x[3] = {o[0] + t * w[0], o[1] + t * w[1], o[2] + t * w[2]};
    int v[3] = {grid_index(g, res, 0, x[0]), grid_index(g, res, 1, x[1]), grid_index(g, res, 2, x[2])};
    double md = INFINITY, mt = INFINITY;
    if (!dda_next(g, bits, res, o, w, v, tf, t_entry, &md, &mt)) return 0;
    for (int a = 0; a < 3; a++) vox[a] = v[a];
    return 1;
}

typedef struct {
    double rgb[3], depth, normal[3];
    int32_t cell, hit, steps, by_max_steps;
    double m_d, m_t, m_x, m_dda; /* decision margins */
} ko_ray_out;

/* Sphere-trace one ray (Sec. 3.4.1).  occ may be NULL.
 * delta_step > 0 switches on conditioning-aware margins: the oracle then also evaluates grad d at
 * every step and propagates a predicted deviation E of a less precise trajectory,
 * E_{k+1} = |1 + grad d(x_k) . w| E_k + delta_step (the step map t -> t + d(t) has slope 1 + grad d . w),
 * and subtracts it from each margin: |d| vs eps loses |grad d . w| E_k, faces and t_far lose E_k. */
void ko_trace_cond(const ko_desc *g, const float *weights, const uint64_t *occ, const double o[3],
                   const double w[3], int max_steps, double eps, double delta_step, ko_ray_out *r) {
    memset(r, 0, sizeof(*r));
    r->depth = INFINITY;
    r->cell = -1;
    r->m_d = r->m_t = r->m_x = r->m_dda = INFINITY;
    double tn, tf;
    if (!ko_clip(g, o, w, &tn, &tf, &r->m_t)) return;
    double t = tn;
    int res = g->occ_res;
    double E = delta_step > 0 ? 0.5 * delta_step : 0.0; /* predicted deviation of t */
    for (int k = 0; k < max_steps; k++) {
        double x[3] = {o[0] + t * w[0], o[1] + t * w[1], o[2] + t * w[2]};
        int cell;
        if (occ) {
            int v[3] = {grid_index(g, res, 0, x[0]), grid_index(g, res, 1, x[1]), grid_index(g, res, 2, x[2])};
            r->m_x = fmin(r->m_x, interior_face_distance(g, res, x) - E);
            if (!occ_test(occ, res, v[0], v[1], v[2])) {
                double te;
                if (!dda_next(g, occ, res, o, w, v, tf, &te, &r->m_dda, &r->m_t)) return; /* miss */
                /* evaluate at the entry face of the voxel the DDA reached; its cell is
                   known exactly from the voxel index, so no floor is taken on the face */
                t = te;
                x[0] = o[0] + t * w[0];
                x[1] = o[1] + t * w[1];
                x[2] = o[2] + t * w[2];
                int f = res / g->N;
                cell = v[0] / f + g->N * (v[1] / f + g->N * (v[2] / f));
            } else {
                cell = ko_cell(g, x);
                r->m_x = fmin(r->m_x, interior_face_distance(g, g->N, x) - E);
            }
        } else {
            cell = ko_cell(g, x);
            r->m_x = fmin(r->m_x, interior_face_distance(g, g->N, x) - E);
        }
        double gw = 0.0;
        double d;
        if (delta_step > 0) {
            double gr[3];
            d = ko_sdf_eval(g, weights, cell, x, NULL, gr);
            gw = gr[0] * w[0] + gr[1] * w[1] + gr[2] * w[2];
        } else {
            d = ko_sdf_eval(g, weights, cell, x, NULL, NULL);
        }
        r->steps++;
        r->m_d = fmin(r->m_d, fabs(fabs(d) - eps) - fabs(gw) * E);
        if (fabs(d) < eps) {
            double feat[KO_MAXIN], grad[3], nrm = 0;
            ko_sdf_eval(g, weights, cell, x, feat, grad);
            for (int c = 0; c < 3; c++) nrm += grad[c] * grad[c];
            nrm = sqrt(nrm);
            for (int c = 0; c < 3; c++) r->normal[c] = nrm > 0 ? grad[c] / nrm : 0.0;
            ko_colour_eval(g, weights, cell, x, feat, r->normal, w, r->rgb);
            r->depth = t;
            r->cell = cell;
            r->hit = 1;
            return;
        }
        t += d;
        if (delta_step > 0) E = fabs(1.0 + gw) * E + delta_step;
        r->m_t = fmin(r->m_t, fmin(fabs(t - tf), fabs(t - tn)) - E);
        if (t > tf || t < tn) return; /* left the box interval [t_near, t_far] */
    }
    r->by_max_steps = 1;
}

void ko_trace(const ko_desc *g, const float *weights, const uint64_t *occ, const double o[3], const double w[3],
              int max_steps, double eps, ko_ray_out *r) {
    ko_trace_cond(g, weights, occ, o, w, max_steps, eps, 0.0, r);
}

/* Render selected pixels.  sel: n_sel global pixel ids (cam*H*W + i*W + j), or NULL for all.
 * Outputs are per selected ray; any output pointer may be NULL. margins: 4 doubles per ray. */
void ko_render(const ko_desc *g, const float *weights, const uint64_t *occ, const float *cams, int n_cams, int W,
               int H, int max_steps, double eps, double delta_step, int64_t n_sel, const int64_t *sel, float *rgb,
               float *depth, float *normal, int32_t *cell, uint8_t *hit, int32_t *steps, double *margins,
               uint8_t *by_max) {
    int64_t n = sel ? n_sel : (int64_t)n_cams * W * H;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < n; q++) {
        int64_t id = sel ? sel[q] : q;
        int64_t cam = id / ((int64_t)W * H), pix = id % ((int64_t)W * H);
        int i = (int)(pix / W), j = (int)(pix % W);
        double o[3], w[3];
        ko_ray(cams + 16 * cam, i, j, o, w);
        ko_ray_out r;
        ko_trace_cond(g, weights, occ, o, w, max_steps, eps, delta_step, &r);
        if (rgb)
            for (int c = 0; c < 3; c++) rgb[3 * q + c] = (float)r.rgb[c];
        if (depth) depth[q] = (float)r.depth;
        if (normal)
            for (int c = 0; c < 3; c++) normal[3 * q + c] = (float)r.normal[c];
        if (cell) cell[q] = r.cell;
        if (hit) hit[q] = (uint8_t)r.hit;
        if (steps) steps[q] = r.steps;
        if (margins) {
            margins[4 * q + 0] = r.m_d;
            margins[4 * q + 1] = r.m_t;
            margins[4 * q + 2] = r.m_x;
            margins[4 * q + 3] = r.m_dda;
        }
        if (by_max) by_max[q] = (uint8_t)r.by_max_steps;
    }
}

/* Same as ko_render but returns depth in double (for pins that need more than FP32). */
void ko_trace_rays(const ko_desc *g, const float *weights, const uint64_t *occ, int64_t n, const double *o,
                   const double *w, int max_steps, double eps, double *depth, int32_t *cell, int32_t *steps,
                   double *normal, double *rgb) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < n; q++) {
        ko_ray_out r;
        ko_trace(g, weights, occ, o + 3 * q, w + 3 * q, max_steps, eps, &r);
        depth[q] = r.depth;
        if (cell) cell[q] = r.cell;
        if (steps) steps[q] = r.steps;
        if (normal)
            for (int c = 0; c < 3; c++) normal[3 * q + c] = r.normal[c];
        if (rgb)
            for (int c = 0; c < 3; c++) rgb[3 * q + c] = r.rgb[c];
    }
}

/* Brute force: march t in [t0, t1] with step dt; at the first sign change of d relative to d(t0)
 * bisect to |interval| < tol.  Returns the root or NAN if none. */
double ko_march_root(const ko_desc *g, const float *weights, const double o[3], const double w[3], double t0,
                     double t1, double dt, double tol) {
    double x[3] = {o[0] + t0 * w[0], o[1] + t0 * w[1], o[2] + t0 * w[2]};
    double d0 = ko_sdf_eval(g, weights, ko_cell(g, x), x, NULL, NULL);
    int s0 = d0 > 0;
    double a = t0;
    for (int64_t k = 1;; k++) {
        double b = t0 + (double)k * dt;
        if (b > t1) b = t1;
        double y[3] = {o[0] + b * w[0], o[1] + b * w[1], o[2] + b * w[2]};
        double d = ko_sdf_eval(g, weights, ko_cell(g, y), y, NULL, NULL);
        if ((d > 0) != s0) {
            while (b - a > tol) {
                double m = 0.5 * (a + b);
                double z[3] = {o[0] + m * w[0], o[1] + m * w[1], o[2] + m * w[2]};
                double dm = ko_sdf_eval(g, weights, ko_cell(g, z), z, NULL, NULL);
                if ((dm > 0) == s0)
                    a = m;
                else
                    b = m;
            }
            return 0.5 * (a + b);
        }
        if (b >= t1) return NAN;
        a = b;
    }
}

void ko_march_roots(const ko_desc *g, const float *weights, int64_t n, const double *o, const double *w,
                    const double *t0, const double *t1, double dt, double tol, double *roots) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < n; q++) roots[q] = ko_march_root(g, weights, o + 3 * q, w + 3 * q, t0[q], t1[q], dt, tol);
}

int ko_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------------------------
 * NeuS-style training loss (Sec. 3.2.2: photometric L1 colour loss over sampled pixels, eikonal
 * regulariser, total L = L_color + lambda L_eik), with the finite-difference gradients of Sec. 3.3.
 *
 * Per ray (origin o, unit direction w, target I): clip to the box; Ns stratified samples
 * t_i = tn + (i + u_i)/Ns (tf - tn); a coarse pass evaluates d at them and forms the NeuS weights
 * T_i alpha_i with alpha_i = max((Phi(d_i) - Phi(d_{i+1})) / Phi(d_i), 0), Phi(d) = sigmoid(s_up d),
 * T_i = prod_{j<i} (1 - alpha_j); Ni importance samples are drawn by inverting the CDF of the
 * piecewise-constant density (T_i alpha_i + 1e-5 on [t_i, t_{i+1}]) at the sorted uniforms u'.
 * All Ns + Ni samples, merged in order, are rendered: d_i and z_i of the cell at x_i, the normal
 * n_i = g_i / |g_i| with g_i the central difference (d(x+h e_k) - d(x-h e_k)) / 2h (each point
 * evaluated in its own cell), colour c_i = sigmoid(colour MLP(z_i, n_i, gamma(w))), alpha_i with
 * Phi(d) = sigmoid(s d), C = sum_i T_i alpha_i c_i.  L_color = (1/B) sum_rays sum_ch |C - I|.
 * Eikonal on M points p: L_eik = (1/M) sum (|g(p)| - 1)^2 with the same central difference.
 * Rays that miss the box render C = 0.  If t_fixed is given, the Ns + Ni sample positions of every
 * ray are taken from it (positions are not differentiated: they are held fixed when the loss is
 * differentiated).  t_out and rgb_out (nullable) receive the positions and the rendered colours C.
 * ------------------------------------------------------------------------------------------- */
static double sdf_at(const ko_desc *g, const float *weights, const double x[3], double *feat) {
    return ko_sdf_eval(g, weights, ko_cell(g, x), x, feat, NULL);
}

static void fd_grad(const ko_desc *g, const float *weights, const double x[3], double h, double gr[3]) {
    for (int k = 0; k < 3; k++) {
        double xp[3] = {x[0], x[1], x[2]}, xm[3] = {x[0], x[1], x[2]};
        xp[k] += h;
        xm[k] -= h;
        gr[k] = (sdf_at(g, weights, xp, NULL) - sdf_at(g, weights, xm, NULL)) / (2.0 * h);
    }
}

double ko_train_loss(const ko_desc *g, const float *weights, double s, double s_up, int64_t B, const double *o,
                     const double *w, const double *target, int Ns, const double *u_s, int Ni, const double *u_i,
                     int64_t M, const double *P, double lambda, double h, const double *t_fixed, double *t_out,
                     double *parts, double *rgb_out) {
    const int S = Ns + Ni;
    double l1 = 0.0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : l1)
    for (int64_t r = 0; r < B; r++) {
        const double *ro = o + 3 * r, *rw = w + 3 * r;
        double tn, tf, margin = INFINITY, C[3] = {0, 0, 0};
        double *ts = (double *)malloc(sizeof(double) * (size_t)S);
        int ok = ko_clip(g, ro, rw, &tn, &tf, &margin);
        if (ok) {
            if (t_fixed) {
                for (int i = 0; i < S; i++) ts[i] = t_fixed[r * S + i];
            } else {
                double *tc = (double *)malloc(sizeof(double) * (size_t)Ns);
                double *dc = (double *)malloc(sizeof(double) * (size_t)Ns);
                double *cdf = (double *)malloc(sizeof(double) * (size_t)Ns);
                for (int i = 0; i < Ns; i++) {
                    tc[i] = tn + ((double)i + u_s[r * Ns + i]) / Ns * (tf - tn);
                    double x[3] = {ro[0] + tc[i] * rw[0], ro[1] + tc[i] * rw[1], ro[2] + tc[i] * rw[2]};
                    dc[i] = sdf_at(g, weights, x, NULL);
                }
                /* coarse weights on the Ns-1 intervals, then their CDF */
                double T = 1.0, tot = 0.0;
                cdf[0] = 0.0;
                for (int i = 0; i + 1 < Ns; i++) {
                    double p0 = 1.0 / (1.0 + exp(-s_up * dc[i])), p1 = 1.0 / (1.0 + exp(-s_up * dc[i + 1]));
                    double a = fmax((p0 - p1) / p0, 0.0);
                    double wgt = T * a + 1e-5;
                    T *= 1.0 - a;
                    tot += wgt;
                    cdf[i + 1] = tot;
                }
                for (int i = 1; i < Ns; i++) cdf[i] /= tot;
                /* inverse CDF at the sorted uniforms, merged with the stratified samples */
                int a = 0, b = 0, k = 0;
                while (a < Ns || b < Ni) {
                    double timp = INFINITY;
                    if (b < Ni) {
                        double u = u_i[r * Ni + b];
                        int j = 0;
                        while (j + 2 < Ns && cdf[j + 1] <= u) j++;
                        double den = cdf[j + 1] - cdf[j];
                        timp = tc[j] + (den > 0 ? (u - cdf[j]) / den : 0.0) * (tc[j + 1] - tc[j]);
                    }
                    if (a < Ns && (b >= Ni || tc[a] <= timp)) {
                        ts[k++] = tc[a++];
                    } else {
                        ts[k++] = timp;
                        b++;
                    }
                }
                free(tc);
                free(dc);
                free(cdf);
            }
            if (t_out)
                for (int i = 0; i < S; i++) t_out[r * S + i] = ts[i];
            double *d = (double *)malloc(sizeof(double) * (size_t)S);
            double (*col)[3] = malloc(sizeof(double) * 3 * (size_t)S);
            for (int i = 0; i < S; i++) {
                double x[3] = {ro[0] + ts[i] * rw[0], ro[1] + ts[i] * rw[1], ro[2] + ts[i] * rw[2]};
                double feat[KO_MAXIN], gr[3], n[3];
                int c = ko_cell(g, x);
                d[i] = ko_sdf_eval(g, weights, c, x, feat, NULL);
                fd_grad(g, weights, x, h, gr);
                double gn = sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
                for (int q = 0; q < 3; q++) n[q] = gn > 0 ? gr[q] / gn : 0.0;
                ko_colour_eval(g, weights, c, x, feat, n, rw, col[i]);
            }
            double T = 1.0;
            for (int i = 0; i + 1 < S; i++) {
                double p0 = 1.0 / (1.0 + exp(-s * d[i])), p1 = 1.0 / (1.0 + exp(-s * d[i + 1]));
                double a = fmax((p0 - p1) / p0, 0.0);
                for (int q = 0; q < 3; q++) C[q] += T * a * col[i][q];
                T *= 1.0 - a;
            }
            free(d);
            free(col);
        } else if (t_out) {
            for (int i = 0; i < S; i++) t_out[r * S + i] = 0.0;
        }
        free(ts);
        for (int q = 0; q < 3; q++) l1 += fabs(C[q] - target[3 * r + q]);
        if (rgb_out)
            for (int q = 0; q < 3; q++) rgb_out[3 * r + q] = C[q];
    }
    double eik = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : eik)
    for (int64_t m = 0; m < M; m++) {
        double gr[3];
        fd_grad(g, weights, P + 3 * m, h, gr);
        double gn = sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
        eik += (gn - 1.0) * (gn - 1.0);
    }
    const double lc = B > 0 ? l1 / (double)B : 0.0, le = M > 0 ? eik / (double)M : 0.0;
    if (parts) {
        parts[0] = lc;
        parts[1] = le;
    }
    return lc + lambda * le;
}

/* ---------------------------------------------------------------------------------------------
 * Reverse-mode gradient of ko_train_loss with respect to every weight of the canonical array.
 * The sample positions are held fixed (they are not differentiated).  |.| and max(., 0) take the
 * derivative 0 at their kinks.  grad (n_cells x params_cell doubles) is overwritten.
 * ------------------------------------------------------------------------------------------- */

/* gradient of (dd * d + sum_k dz[k] z[k]) at x in `cell` with respect to the cell's SDF weights
 * (accumulated into gw, which points at the cell's first weight) */
static void sdf_backward(const ko_desc *g, const float *weights, int cell, const double x[3], double dd,
                         const double *dz, double *gw) {
    int dims[KO_MAXLAYERS + 2];
    int nd = sdf_dims(g, dims);
    int nl = nd - 1;
    const float *w = weights + (int64_t)cell * ko_params_cell(g);
    double act[KO_MAXLAYERS + 1][KO_MAXIN], pre[KO_MAXLAYERS][KO_MAXW];
    int64_t offs[KO_MAXLAYERS];
    int64_t off = 0;
    for (int l = 0; l < nl; l++) {
        offs[l] = off;
        off += (int64_t)dims[l] * dims[l + 1] + dims[l + 1];
    }
    ko_pe(g->pe_pos_L, 3, x, act[0]);
    for (int l = 0; l < nl; l++) {
        const float *W = w + offs[l], *b = W + (int64_t)dims[l] * dims[l + 1];
        for (int o = 0; o < dims[l + 1]; o++) {
            double s = (double)b[o];
            for (int i = 0; i < dims[l]; i++) s += (double)W[(int64_t)o * dims[l] + i] * act[l][i];
            pre[l][o] = s;
            act[l + 1][o] = (l + 1 < nl) ? ko_softplus(s, g->beta) : s;
        }
    }
    /* delta = dL / d pre[l] */
    double delta[KO_MAXIN], nxt[KO_MAXIN];
    delta[0] = dd;
    for (int k = 0; k < g->feat_dim; k++) delta[1 + k] = dz ? dz[k] : 0.0;
    for (int l = nl - 1; l >= 0; l--) {
        const float *W = w + offs[l];
        double *gW = gw + offs[l], *gb = gW + (int64_t)dims[l] * dims[l + 1];
        for (int o = 0; o < dims[l + 1]; o++) {
            gb[o] += delta[o];
            for (int i = 0; i < dims[l]; i++) gW[(int64_t)o * dims[l] + i] += delta[o] * act[l][i];
        }
        if (l == 0) break;
        for (int i = 0; i < dims[l]; i++) {
            double s = 0;
            for (int o = 0; o < dims[l + 1]; o++) s += (double)W[(int64_t)o * dims[l] + i] * delta[o];
            nxt[i] = s * dsoftplus(pre[l - 1][i], g->beta);
        }
        memcpy(delta, nxt, sizeof(double) * dims[l]);
    }
}

/* gradient of drgb . rgb (rgb = colour MLP output) with respect to the cell's colour weights
 * (accumulated into gw, which points at the cell's first colour weight) and to the inputs feat and n */
static void colour_backward(const ko_desc *g, const float *weights, int cell, const double x[3], const double *feat,
                            const double n[3], const double v[3], const double drgb[3], double *gw, double *dfeat,
                            double dn[3]) {
    int dims[KO_MAXLAYERS + 2];
    int nd = col_dims(g, dims);
    int nl = nd - 1;
    const float *w = weights + (int64_t)cell * ko_params_cell(g) + ko_params_sdf(g);
    double act[KO_MAXLAYERS + 1][KO_MAXIN], pre[KO_MAXLAYERS][KO_MAXW];
    int64_t offs[KO_MAXLAYERS];
    int64_t off = 0;
    for (int l = 0; l < nl; l++) {
        offs[l] = off;
        off += (int64_t)dims[l] * dims[l + 1] + dims[l + 1];
    }
    int u = 0;
    for (int k = 0; k < g->feat_dim; k++) act[0][u++] = feat[k];
    for (int c = 0; c < 3; c++) act[0][u++] = n[c];
    ko_pe(g->pe_dir_L, 3, v, act[0] + u);
    u += 3 + 6 * g->pe_dir_L;
    if (g->col_use_x)
        for (int c = 0; c < 3; c++) act[0][u++] = x[c];
    for (int l = 0; l < nl; l++) {
        const float *W = w + offs[l], *b = W + (int64_t)dims[l] * dims[l + 1];
        for (int o = 0; o < dims[l + 1]; o++) {
            double s = (double)b[o];
            for (int i = 0; i < dims[l]; i++) s += (double)W[(int64_t)o * dims[l] + i] * act[l][i];
            pre[l][o] = s;
            act[l + 1][o] = (l + 1 < nl) ? fmax(s, 0.0) : sigmoid(s);
        }
    }
    double delta[KO_MAXIN], nxt[KO_MAXIN];
    for (int c = 0; c < 3; c++) delta[c] = drgb[c] * act[nl][c] * (1.0 - act[nl][c]);
    for (int l = nl - 1; l >= 0; l--) {
        const float *W = w + offs[l];
        double *gW = gw + offs[l], *gb = gW + (int64_t)dims[l] * dims[l + 1];
        for (int o = 0; o < dims[l + 1]; o++) {
            gb[o] += delta[o];
            for (int i = 0; i < dims[l]; i++) gW[(int64_t)o * dims[l] + i] += delta[o] * act[l][i];
        }
        for (int i = 0; i < dims[l]; i++) {
            double s = 0;
            for (int o = 0; o < dims[l + 1]; o++) s += (double)W[(int64_t)o * dims[l] + i] * delta[o];
            nxt[i] = (l > 0) ? (pre[l - 1][i] > 0 ? s : 0.0) : s;
        }
        memcpy(delta, nxt, sizeof(double) * dims[l]);
    }
    for (int k = 0; k < g->feat_dim; k++) dfeat[k] = delta[k];
    for (int c = 0; c < 3; c++) dn[c] = delta[g->feat_dim + c];
}

/* the six central-difference points around x get upstream +-dgr[k] / 2h */
static void fd_backward(const ko_desc *g, const float *weights, const double x[3], double h, const double dgr[3],
                        double *grad, int64_t pc) {
    for (int k = 0; k < 3; k++) {
        double xp[3] = {x[0], x[1], x[2]}, xm[3] = {x[0], x[1], x[2]};
        xp[k] += h;
        xm[k] -= h;
        int cp = ko_cell(g, xp), cm = ko_cell(g, xm);
        sdf_backward(g, weights, cp, xp, dgr[k] / (2.0 * h), NULL, grad + (int64_t)cp * pc);
        sdf_backward(g, weights, cm, xm, -dgr[k] / (2.0 * h), NULL, grad + (int64_t)cm * pc);
    }
}

double ko_train_grad(const ko_desc *g, const float *weights, double s, double s_up, int64_t B, const double *o,
                     const double *w, const double *target, int Ns, const double *u_s, int Ni, const double *u_i,
                     int64_t M, const double *P, double lambda, double h, const double *t_fixed, double *grad,
                     double *parts) {
    const int S = Ns + Ni;
    const int64_t pc = ko_params_cell(g), ncell = (int64_t)g->N * g->N * g->N, nw = pc * ncell;
    const int64_t psdf = ko_params_sdf(g);
    double *ts = (double *)malloc(sizeof(double) * (size_t)(B > 0 ? B : 1) * S);
    double loss = ko_train_loss(g, weights, s, s_up, B, o, w, target, Ns, u_s, Ni, u_i, M, P, lambda, h, t_fixed,
                                ts, parts, NULL);
    memset(grad, 0, sizeof(double) * (size_t)nw);
    /* serial accumulation keeps the oracle plain; it is sized for test problems */
    for (int64_t r = 0; r < B; r++) {
        const double *ro = o + 3 * r, *rw = w + 3 * r;
        double tn, tf, margin = INFINITY;
        if (!ko_clip(g, ro, rw, &tn, &tf, &margin)) continue;
        const double *t = ts + r * S;
        double *d = malloc(sizeof(double) * S), *Phi = malloc(sizeof(double) * S), *alpha = malloc(sizeof(double) * S);
        double *Tr = malloc(sizeof(double) * S), (*col)[3] = malloc(sizeof(double) * 3 * S);
        double (*feat)[KO_MAXIN] = malloc(sizeof(double) * KO_MAXIN * S), (*nrm)[3] = malloc(sizeof(double) * 3 * S);
        double *gnorm = malloc(sizeof(double) * S), (*gr)[3] = malloc(sizeof(double) * 3 * S);
        int *cell = malloc(sizeof(int) * S);
        for (int i = 0; i < S; i++) {
            double x[3] = {ro[0] + t[i] * rw[0], ro[1] + t[i] * rw[1], ro[2] + t[i] * rw[2]};
            cell[i] = ko_cell(g, x);
            d[i] = ko_sdf_eval(g, weights, cell[i], x, feat[i], NULL);
            fd_grad(g, weights, x, h, gr[i]);
            gnorm[i] = sqrt(gr[i][0] * gr[i][0] + gr[i][1] * gr[i][1] + gr[i][2] * gr[i][2]);
            for (int q = 0; q < 3; q++) nrm[i][q] = gnorm[i] > 0 ? gr[i][q] / gnorm[i] : 0.0;
            ko_colour_eval(g, weights, cell[i], x, feat[i], nrm[i], rw, col[i]);
            Phi[i] = 1.0 / (1.0 + exp(-s * d[i]));
        }
        double T = 1.0, C[3] = {0, 0, 0};
        for (int i = 0; i + 1 < S; i++) {
            alpha[i] = fmax((Phi[i] - Phi[i + 1]) / Phi[i], 0.0);
            Tr[i] = T;
            for (int q = 0; q < 3; q++) C[q] += T * alpha[i] * col[i][q];
            T *= 1.0 - alpha[i];
        }
        double gC[3];
        for (int q = 0; q < 3; q++) {
            double e = C[q] - target[3 * r + q];
            gC[q] = (e > 0 ? 1.0 : (e < 0 ? -1.0 : 0.0)) / (double)B;
        }
        /* Chat = colour rendered from sample i+1 on with unit transmittance, built back to front */
        double Chat[3] = {0, 0, 0};
        double *dd = calloc((size_t)S, sizeof(double));
        for (int i = S - 2; i >= 0; i--) {
            double dalpha = 0.0;
            for (int q = 0; q < 3; q++) dalpha += Tr[i] * gC[q] * (col[i][q] - Chat[q]);
            if ((Phi[i] - Phi[i + 1]) / Phi[i] > 0) {
                dd[i] += dalpha * s * Phi[i + 1] * (1.0 - Phi[i]) / Phi[i];
                dd[i + 1] -= dalpha * s * Phi[i + 1] * (1.0 - Phi[i + 1]) / Phi[i];
            }
            for (int q = 0; q < 3; q++) Chat[q] = alpha[i] * col[i][q] + (1.0 - alpha[i]) * Chat[q];
        }
        for (int i = 0; i < S; i++) {
            double x[3] = {ro[0] + t[i] * rw[0], ro[1] + t[i] * rw[1], ro[2] + t[i] * rw[2]};
            double dz[KO_MAXIN] = {0}, dn[3] = {0, 0, 0};
            if (i + 1 < S) {
                double drgb[3];
                for (int q = 0; q < 3; q++) drgb[q] = Tr[i] * alpha[i] * gC[q];
                colour_backward(g, weights, cell[i], x, feat[i], nrm[i], rw, drgb, grad + cell[i] * pc + psdf, dz,
                                dn);
            }
            sdf_backward(g, weights, cell[i], x, dd[i], dz, grad + cell[i] * pc);
            if (gnorm[i] > 0) {
                double nd = nrm[i][0] * dn[0] + nrm[i][1] * dn[1] + nrm[i][2] * dn[2], dgr[3];
                for (int q = 0; q < 3; q++) dgr[q] = (dn[q] - nrm[i][q] * nd) / gnorm[i];
                fd_backward(g, weights, x, h, dgr, grad, pc);
            }
        }
        free(dd);
        free(d);
        free(Phi);
        free(alpha);
        free(Tr);
        free(col);
        free(feat);
        free(nrm);
        free(gnorm);
        free(gr);
        free(cell);
    }
    for (int64_t m = 0; m < M; m++) {
        double gm[3];
        fd_grad(g, weights, P + 3 * m, h, gm);
        double gn = sqrt(gm[0] * gm[0] + gm[1] * gm[1] + gm[2] * gm[2]);
        if (gn <= 0) continue;
        double dgr[3];
        for (int q = 0; q < 3; q++) dgr[q] = lambda / (double)M * 2.0 * (gn - 1.0) * gm[q] / gn;
        fd_backward(g, weights, P + 3 * m, h, dgr, grad, pc);
    }
    free(ts);
    return loss;
}

/* ---------------------------------------------------------------------------------------------
 * Lambertian path tracing of the KiloNeuS surface (Sec. 3.4: the path tracer treats the surface as
 * Lambertian; the colour network gives its albedo, the normalised SDF gradient its normal).
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the k-th output of the generator
 * seeded with s is mix(s + (k + 1) * 0x9E3779B97F4A7C15); a uniform in [0, 1) is its top 24 bits
 * times 2^-24 (exact in float and double).  Path p, trace depth t, dimension i use k = (p * 16 + t)
 * * 4 + i.
 * Path p of pixel (c, i, j) and sample s: p = ((c * H + i) * W + j) * spp + s.  Its primary ray goes
 * through the point (j + u_0, i + u_1) of the image plane (u from depth 0).  At each depth the ray is
 * sphere-traced (ko_trace); a miss adds beta * E(w) and ends the path, E(w) = (1 - a) horizon +
 * a zenith with a = (w_z + 1) / 2; a hit multiplies beta by the albedo (the colour MLP at the hit,
 * seen from the ray) and, below the last depth, continues from x + offset * n in a cosine-weighted
 * direction about n (u_2, u_3 of this depth; orthonormal basis of Duff et al., JCGT 2017); a hit at
 * the last depth ends the path with no light.  Pixel value = mean over its spp paths.
 * ------------------------------------------------------------------------------------------- */
#define KO_PT_MAXDEPTH 16

uint64_t ko_splitmix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double ko_pt_uniform(uint64_t seed, int64_t path, int depth, int dim) {
    uint64_t k = ((uint64_t)path * KO_PT_MAXDEPTH + (uint64_t)depth) * 4u + (uint64_t)dim;
    return (double)(ko_splitmix64(seed, k) >> 40) * 0x1p-24;
}

/* cosine-weighted unit direction about the unit normal n */
void ko_cosine_dir(const double n[3], double u1, double u2, double w[3]) {
    double sign = n[2] >= 0 ? 1.0 : -1.0;
    double a = -1.0 / (sign + n[2]);
    double b = n[0] * n[1] * a;
    double t[3] = {1.0 + sign * n[0] * n[0] * a, sign * b, -sign * n[0]};
    double bb[3] = {b, sign + n[1] * n[1] * a, -n[1]};
    double r = sqrt(u2), phi = 2.0 * M_PI * u1, z = sqrt(1.0 - u2);
    for (int k = 0; k < 3; k++) w[k] = r * cos(phi) * t[k] + r * sin(phi) * bb[k] + z * n[k];
}

void ko_sky(const double w[3], const double horizon[3], const double zenith[3], double out[3]) {
    double a = 0.5 * (w[2] + 1.0);
    for (int k = 0; k < 3; k++) out[k] = (1.0 - a) * horizon[k] + a * zenith[k];
}

/* path tracing of the selected pixels; L (n_sel * spp * 3) and traces (n_sel * spp) per path are
 * optional outputs */
void ko_path_trace(const ko_desc *g, const float *weights, const uint64_t *occ, const float *cams, int n_cams,
                   int W, int H, int spp, int max_depth, int max_steps, double eps, double offset, uint64_t seed,
                   const double *horizon, const double *zenith, int64_t n_sel, const int64_t *sel, double *rgb,
                   double *L_out, int32_t *traces_out) {
    if (max_depth > KO_PT_MAXDEPTH) max_depth = KO_PT_MAXDEPTH;
    (void)n_cams;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < n_sel; q++) {
        const int64_t pix = sel[q];
        const int c = (int)(pix / ((int64_t)W * H));
        const int i = (int)((pix / W) % H), j = (int)(pix % W);
        const float *cam = cams + 16 * c;
        double acc[3] = {0, 0, 0};
        for (int s = 0; s < spp; s++) {
            const int64_t path = pix * spp + s;
            double o[3], w[3], beta[3] = {1, 1, 1}, L[3] = {0, 0, 0};
            {
                double u0 = ko_pt_uniform(seed, path, 0, 0), u1 = ko_pt_uniform(seed, path, 0, 1);
                double dc[3] = {((double)j + u0 - cam[14]) / cam[12], ((double)i + u1 - cam[15]) / cam[13], 1.0};
                double nrm = 0;
                for (int r = 0; r < 3; r++) {
                    w[r] = cam[4 * r + 0] * dc[0] + cam[4 * r + 1] * dc[1] + cam[4 * r + 2] * dc[2];
                    nrm += w[r] * w[r];
                    o[r] = cam[4 * r + 3];
                }
                nrm = sqrt(nrm);
                for (int r = 0; r < 3; r++) w[r] /= nrm;
            }
            int traces = 0;
            for (int depth = 0; depth < max_depth; depth++) {
                ko_ray_out r;
                ko_trace(g, weights, occ, o, w, max_steps, eps, &r);
                traces++;
                if (!r.hit) {
                    double e[3];
                    ko_sky(w, horizon, zenith, e);
                    for (int k = 0; k < 3; k++) L[k] += beta[k] * e[k];
                    break;
                }
                for (int k = 0; k < 3; k++) beta[k] *= r.rgb[k];
                if (depth + 1 == max_depth) break;
                double x[3], nw[3];
                for (int k = 0; k < 3; k++) x[k] = o[k] + r.depth * w[k] + offset * r.normal[k];
                ko_cosine_dir(r.normal, ko_pt_uniform(seed, path, depth, 2), ko_pt_uniform(seed, path, depth, 3), nw);
                for (int k = 0; k < 3; k++) {
                    o[k] = x[k];
                    w[k] = nw[k];
                }
            }
            for (int k = 0; k < 3; k++) acc[k] += L[k];
            if (L_out)
                for (int k = 0; k < 3; k++) L_out[3 * (q * spp + s) + k] = L[k];
            if (traces_out) traces_out[q * spp + s] = traces;
        }
        for (int k = 0; k < 3; k++) rgb[3 * q + k] = acc[k] / spp;
    }
}

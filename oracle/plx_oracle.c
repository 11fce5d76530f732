/*
 * plx_oracle.c -- plain FP64 CPU oracle for the Plenoxels differentiable
 * volume renderer (Yu, Fridovich-Keil et al., "Plenoxels: Radiance Fields
 * without Neural Networks", arXiv 2112.05131).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * constant with the CUDA library in paper_2112_05131_gb300/csrc; the two are
 * compared element by element on the same seeded inputs.
 *
 * Everything here is written for a reader checking it against the paper by
 * eye: one loop per definition, FP64 arithmetic, no blocking, no skipping of
 * empty space, no early exits other than the ones the definition states.
 *
 * Grid semantics (Sec. 3.2; Supp. B.1):
 *   - a dense int32 index volume idx[R*R*R]; idx[n] == -1 is a NULL cell,
 *     otherwise it is the row of that node in the data table;
 *   - node (i,j,k) has linear id n = (i*R + j)*R + k (k fastest, i <-> x);
 *   - a data row holds 28 values [sigma, R0..R8, G0..G8, B0..B8] at
 *     `row_stride` doubles per row (28 or more; FP32 inputs convert exactly);
 *   - NULL cells count as all-zero values (Supp. B.1);
 *   - values live on the lattice nodes, the voxel corners (Sec. 3);
 *     node (i,j,k) sits at aabb_min + (i,j,k) * h, h = (aabb_max-aabb_min)/(R-1).
 *
 * Parity status of each function (what pins it, in tests/test_oracle_pins.py):
 *   orc_sh_basis        pinned: quadrature orthonormality, textbook values
 *   orc_interp          pinned: affine fields reproduced exactly; hat-function
 *                       brute force on 4^3
 *   orc_gen_rays        pinned: pixel-centre geometry of hand-built cameras
 *   orc_clip            pinned: axis-aligned and diagonal rays with known hits
 *   orc_render          pinned: constant-field closed form exp(-sigma t),
 *                       telescoped (T_i - T_{i+1}) form, brute force on 4^3,
 *                       empty grid = background, sum of weights + T_end = 1
 *   orc_render_backward pinned: central finite differences of orc_render
 *   orc_render_backward_abs  pinned: bounds the adjoint of every smaller g
 *                       (triangle inequality), equals it for one-sign terms
 *   orc_render_backward_mag  pinned: dominates the absolute-value adjoint,
 *                       equals it where T_{s+1} c and R_s do not cancel
 *   orc_tv              pinned: linear-ramp closed form, finite differences
 *   orc_rmsprop         pinned: constant-gradient closed form
 *   orc_max_weight      pinned: closed form exp(-sigma s delta)(1 - exp(-sigma
 *                       delta)) on a constant field along an axis, which also
 *                       fixes the 8-corner attribution; max over a union of
 *                       ray sets = elementwise max; empty grid = all zero
 *   orc_sparsity        pinned: constant-field closed form lambda N log(1 +
 *                       2 sigma0^2) with total gradient lambda N 4 sigma0 /
 *                       (1 + 2 sigma0^2); central finite differences;
 *                       negative densities give zero
 *   orc_prune           pinned: exhaustive 3x3x3 enumeration on small grids
 *   orc_prune_key       pinned: equals orc_prune for key = density; exhaustive
 *                       enumeration with a random key
 *   orc_upsample        pinned: affine field resampled exactly; exhaustive
 *                       support enumeration on small grids
 *   orc_round_bf16      pinned: exact RNE cases (ties, carries) by hand
 *   SH sign/order convention and the learning-rate delay multiplier are
 *   conventions, not facts of the paper: parity unpinned for those choices.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_NV 28 /* 1 density + 3 channels x 9 SH coefficients (Sec. 3.2) */
#define ORC_NSH 9 /* degree-2 real spherical harmonics (Sec. 3.2)          */

/* ------------------------------------------------------------------------- */
/* Real spherical harmonics up to degree 2, orthonormal on the unit sphere.   */
/* Sec. 3.2: colour = sum of SH basis functions weighted by the coefficients. */
/* Order/sign convention (shared with the CUDA path by specification only):   */
/*   Y0 = 1/(2 sqrt(pi))                                                      */
/*   Y1 = -sqrt(3/(4pi)) y, Y2 = sqrt(3/(4pi)) z, Y3 = -sqrt(3/(4pi)) x       */
/*   Y4 = 1/2 sqrt(15/pi) xy, Y5 = -1/2 sqrt(15/pi) yz,                       */
/*   Y6 = 1/4 sqrt(5/pi) (3z^2 - 1), Y7 = -1/2 sqrt(15/pi) xz,                */
/*   Y8 = 1/4 sqrt(15/pi) (x^2 - y^2)                                         */
/* ------------------------------------------------------------------------- */
void orc_sh_basis(const double *dir, double *Y)
{
    const double pi = 3.14159265358979323846;
    double x = dir[0], y = dir[1], z = dir[2];
    Y[0] = 0.5 * sqrt(1.0 / pi);
    Y[1] = -sqrt(3.0 / (4.0 * pi)) * y;
    Y[2] = sqrt(3.0 / (4.0 * pi)) * z;
    Y[3] = -sqrt(3.0 / (4.0 * pi)) * x;
    Y[4] = 0.5 * sqrt(15.0 / pi) * x * y;
    Y[5] = -0.5 * sqrt(15.0 / pi) * y * z;
    Y[6] = 0.25 * sqrt(5.0 / pi) * (3.0 * z * z - 1.0);
    Y[7] = -0.5 * sqrt(15.0 / pi) * x * z;
    Y[8] = 0.25 * sqrt(15.0 / pi) * (x * x - y * y);
}

/* ------------------------------------------------------------------------- */
/* Grid description and NULL-as-zero value lookup (Supp. B.1).               */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t R;
    const int32_t *idx;
    const double *rows;
    int64_t row_stride;
    double lo[3], hi[3], h[3];
} orc_grid;

static void grid_init(orc_grid *g, int64_t R, const int32_t *idx, const double *rows,
                      int64_t row_stride, const double *aabb)
{
    g->R = R;
    g->idx = idx;
    g->rows = rows;
    g->row_stride = row_stride;
    for (int a = 0; a < 3; ++a) {
        g->lo[a] = aabb[a];
        g->hi[a] = aabb[3 + a];
        g->h[a] = (g->hi[a] - g->lo[a]) / (double)(R - 1);
    }
}

static int64_t node_id(int64_t R, int64_t i, int64_t j, int64_t k)
{
    return (i * R + j) * R + k;
}

/* value d of node n; a NULL node has all values 0 */
static double node_value(const orc_grid *g, int64_t n, int d)
{
    int32_t r = g->idx[n];
    if (r < 0) return 0.0;
    return g->rows[(int64_t)r * g->row_stride + d];
}

/* ------------------------------------------------------------------------- */
/* Trilinear interpolation of all 28 values at world point p (Sec. 3.3).     */
/* g = (p - aabb_min)/h clamped to [0, R-1]; base = min(floor(g), R-2);      */
/* f = g - base; corner c = (cx,cy,cz) has weight prod_a (c_a ? f_a : 1-f_a).*/
/* Also returns the 8 corner node ids and weights for the adjoint.           */
/* ------------------------------------------------------------------------- */
static void interp_at(const orc_grid *g, const double p[3], double out[ORC_NV],
                      int64_t corner_node[8], double corner_w[8])
{
    int64_t base[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double ga = (p[a] - g->lo[a]) / g->h[a];
        if (ga < 0.0) ga = 0.0;
        if (ga > (double)(g->R - 1)) ga = (double)(g->R - 1);
        int64_t b = (int64_t)floor(ga);
        if (b > g->R - 2) b = g->R - 2;
        base[a] = b;
        f[a] = ga - (double)b;
    }
    for (int d = 0; d < ORC_NV; ++d) out[d] = 0.0;
    for (int c = 0; c < 8; ++c) {
        int cx = (c >> 2) & 1, cy = (c >> 1) & 1, cz = c & 1;
        double w = (cx ? f[0] : 1.0 - f[0]) * (cy ? f[1] : 1.0 - f[1]) *
                   (cz ? f[2] : 1.0 - f[2]);
        int64_t n = node_id(g->R, base[0] + cx, base[1] + cy, base[2] + cz);
        corner_node[c] = n;
        corner_w[c] = w;
        for (int d = 0; d < ORC_NV; ++d) out[d] += w * node_value(g, n, d);
    }
}

/* Exported: interpolate at n_pts world points; out is [n_pts, 28]. */
void orc_interp(int64_t R, const int32_t *idx, const double *rows, int64_t row_stride,
                const double *aabb, const double *pts, int64_t n_pts, double *out)
{
    orc_grid g;
    grid_init(&g, R, idx, rows, row_stride, aabb);
    int64_t cn[8];
    double cw[8];
    for (int64_t q = 0; q < n_pts; ++q) interp_at(&g, pts + 3 * q, out + ORC_NV * q, cn, cw);
}

/* ------------------------------------------------------------------------- */
/* Ray generation through pixel centres (Sec. 4.1 uses centred pixels;      */
/* Supp. D notes the JAXNeRF centring fix).  Pinhole camera looking down -z, */
/* y up.  cams is [n_cams, 18]: c2w (3x4 row-major), fx, fy, cx, cy, W, H.  */
/* Pixel id p = view*H*W + v*W + u; all cameras share W and H.               */
/* ------------------------------------------------------------------------- */
void orc_gen_rays(const double *cams, const int64_t *pix, int64_t n, double *o, double *d)
{
    int64_t W = (int64_t)cams[16], H = (int64_t)cams[17];
    for (int64_t r = 0; r < n; ++r) {
        int64_t p = pix[r];
        int64_t view = p / (H * W);
        int64_t rem = p - view * H * W;
        int64_t v = rem / W, u = rem - v * W;
        const double *cam = cams + 18 * view;
        double dc[3];
        dc[0] = ((double)u + 0.5 - cam[14]) / cam[12];
        dc[1] = -((double)v + 0.5 - cam[15]) / cam[13];
        dc[2] = -1.0;
        double dw[3], len2 = 0.0;
        for (int i = 0; i < 3; ++i) {
            dw[i] = cam[4 * i + 0] * dc[0] + cam[4 * i + 1] * dc[1] + cam[4 * i + 2] * dc[2];
            len2 += dw[i] * dw[i];
        }
        double inv = 1.0 / sqrt(len2);
        for (int i = 0; i < 3; ++i) {
            d[3 * r + i] = dw[i] * inv;
            o[3 * r + i] = cam[4 * i + 3];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Ray / axis-aligned box clip (slab test).  t_near = max(t_in, 0).          */
/* Returns 1 on a hit (t_far > t_near).                                      */
/* ------------------------------------------------------------------------- */
static int clip_ray(const double o[3], const double d[3], const double lo[3],
                    const double hi[3], double *tn, double *tf)
{
    double t0 = -INFINITY, t1 = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < lo[a] || o[a] > hi[a]) return 0;
            continue;
        }
        double ta = (lo[a] - o[a]) / d[a];
        double tb = (hi[a] - o[a]) / d[a];
        double tmin = ta < tb ? ta : tb;
        double tmax = ta < tb ? tb : ta;
        if (tmin > t0) t0 = tmin;
        if (tmax < t1) t1 = tmax;
    }
    if (t0 < 0.0) t0 = 0.0;
    *tn = t0;
    *tf = t1;
    return t1 > t0;
}

/* Exported clip: out is [n, 3] = (t_near, t_far, hit). */
void orc_clip(const double *o, const double *d, int64_t n, const double *aabb, double *out)
{
    for (int64_t r = 0; r < n; ++r) {
        double tn = 0.0, tf = 0.0;
        int hit = clip_ray(o + 3 * r, d + 3 * r, aabb, aabb + 3, &tn, &tf);
        out[3 * r + 0] = tn;
        out[3 * r + 1] = tf;
        out[3 * r + 2] = hit ? 1.0 : 0.0;
    }
}

/* ------------------------------------------------------------------------- */
/* One sample of the march: everything the adjoint needs.                    */
/* ------------------------------------------------------------------------- */
typedef struct {
    double sigma_pre;     /* interpolated density before the activation      */
    double sigma;         /* max(0, sigma_pre)                               */
    double k[ORC_NV - 1]; /* interpolated SH coefficients, [ch*9 + l]        */
    double pre[3];        /* sum_l Y_l k_{ch,l}                              */
    double c[3];          /* ReLU colour (Supp. B.1)                         */
    double T;             /* transmittance before this sample                */
    double alpha;         /* 1 - exp(-sigma * delta)                         */
    double w;             /* T * alpha                                       */
    int64_t node[8];
    double cw[8];
} orc_sample;

typedef struct {
    double rgb[3];
    double T_end;
    int64_t n_samples;
    double ratio; /* (t_far - t_near) / delta, for sample-count tie flags */
    int hit;
} orc_ray_out;

/*
 * March one ray (Eq. 1, Sec. 3.1).  Samples t_s = t_near + s*delta for
 * s = 0,1,... while t_s < t_far; every sample has delta_s = delta (the
 * distance to the next sample).  Before sample s, if T_s < stop_thresh the
 * march stops and T_end = T_s.  C = sum_s T_s alpha_s c_s + T_end * bg.
 * If `samples` is non-NULL the per-sample state is stored there (capacity
 * `cap`; the march is truncated at `cap`, which callers size generously).
 */
static int64_t march(const orc_grid *g, const double o[3], const double dir[3], double delta,
                     const double bg[3], double stop_thresh, orc_ray_out *res,
                     orc_sample *samples, int64_t cap)
{
    double Y[ORC_NSH];
    orc_sh_basis(dir, Y);
    double tn = 0.0, tf = 0.0;
    int hit = clip_ray(o, dir, g->lo, g->hi, &tn, &tf);
    res->hit = hit;
    res->ratio = hit ? (tf - tn) / delta : 0.0;
    double C[3] = {0.0, 0.0, 0.0};
    double T = 1.0;
    int64_t s = 0;
    if (hit) {
        for (;; ++s) {
            double t = tn + (double)s * delta;
            if (!(t < tf)) break;
            if (T < stop_thresh) break;
            orc_sample smp;
            double p[3], v[ORC_NV];
            for (int a = 0; a < 3; ++a) p[a] = o[a] + t * dir[a];
            interp_at(g, p, v, smp.node, smp.cw);
            smp.sigma_pre = v[0];
            smp.sigma = v[0] > 0.0 ? v[0] : 0.0;
            for (int q = 0; q < ORC_NV - 1; ++q) smp.k[q] = v[1 + q];
            for (int ch = 0; ch < 3; ++ch) {
                double acc = 0.0;
                for (int l = 0; l < ORC_NSH; ++l) acc += Y[l] * v[1 + ch * ORC_NSH + l];
                smp.pre[ch] = acc;
                smp.c[ch] = acc > 0.0 ? acc : 0.0;
            }
            smp.T = T;
            smp.alpha = 1.0 - exp(-smp.sigma * delta);
            smp.w = T * smp.alpha;
            for (int ch = 0; ch < 3; ++ch) C[ch] += smp.w * smp.c[ch];
            T = T * (1.0 - smp.alpha);
            if (samples) {
                if (s >= cap) break;
                samples[s] = smp;
            }
        }
    }
    for (int ch = 0; ch < 3; ++ch) res->rgb[ch] = C[ch] + T * bg[ch];
    res->T_end = T;
    res->n_samples = s;
    return s;
}

/*
 * Exported forward render.  o, d: [n,3] (d unit length, used as given).
 * opts: [step_vox, bg_r, bg_g, bg_b, stop_thresh]; delta = step_vox * min_a h_a.
 * rgb: [n,3].  aux (nullable): [n,4] = (T_end, n_samples, ratio, hit).
 */
void orc_render(int64_t R, const int32_t *idx, const double *rows, int64_t row_stride,
                const double *aabb, const double *o, const double *d, int64_t n,
                const double *opts, double *rgb, double *aux)
{
    orc_grid g;
    grid_init(&g, R, idx, rows, row_stride, aabb);
    double hmin = g.h[0] < g.h[1] ? g.h[0] : g.h[1];
    if (g.h[2] < hmin) hmin = g.h[2];
    double delta = opts[0] * hmin;
    double bg[3] = {opts[1], opts[2], opts[3]};
    double stop = opts[4];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < n; ++r) {
        orc_ray_out res;
        march(&g, o + 3 * r, d + 3 * r, delta, bg, stop, &res, NULL, 0);
        for (int ch = 0; ch < 3; ++ch) rgb[3 * r + ch] = res.rgb[ch];
        if (aux) {
            aux[4 * r + 0] = res.T_end;
            aux[4 * r + 1] = (double)res.n_samples;
            aux[4 * r + 2] = res.ratio;
            aux[4 * r + 3] = (double)res.hit;
        }
    }
}

/*
 * Exported adjoint of orc_render (Sec. 3.5: the renderer is differentiable;
 * Supp. B.1, on its gradient kernels).  grad_rgb [n,3] = dL/dC.  Accumulates
 * (+=) dL/d(row values) into grad_rows [M, 28] (FP64, dense 28 columns).
 *
 * Per sample s, with R_s = sum_{j>s} w_j c_j + T_end bg computed as an
 * explicit suffix sum:
 *   dL/dc_{s,ch}     = g_ch * w_s
 *   dL/dk_{s,ch,l}   = dL/dc_{s,ch} * [pre_{s,ch} > 0] * Y_l
 *   dL/dsigma_s      = delta * sum_ch g_ch (T_{s+1} c_{s,ch} - R_{s,ch})
 *                      * [sigma_pre_s > 0]
 * and each per-sample gradient reaches corner node c with its trilinear
 * weight; NULL corners receive nothing.
 */
/*
 * abs_mode = 1 adds every per-sample, per-corner term in absolute value
 * (|g_ch| and |T_{s+1} c - R_s|, |Y_l| in place of the signed factors): for
 * g >= 0 the result bounds |adjoint(g')| for every g' with |g'| <= g, which
 * the tests use to carry an uncertainty of dL/dC into the gradient.
 * abs_mode = 2 ("magnitude") takes the density term's two operands apart,
 * |g_ch| delta (T_{s+1} |c| + |R_s|): the size of the numbers an FP32
 * implementation subtracts, which bounds its rounding error where they
 * nearly cancel (long rays whose colours resemble what lies behind them).
 */
static void render_backward_impl(int64_t R, const int32_t *idx, const double *rows, int64_t row_stride,
                                 const double *aabb, const double *o, const double *d, int64_t n,
                                 const double *opts, const double *grad_rgb, double *grad_rows, int abs_mode)
{
    orc_grid g;
    grid_init(&g, R, idx, rows, row_stride, aabb);
    double hmin = g.h[0] < g.h[1] ? g.h[0] : g.h[1];
    if (g.h[2] < hmin) hmin = g.h[2];
    double delta = opts[0] * hmin;
    double bg[3] = {opts[1], opts[2], opts[3]};
    double stop = opts[4];
    /* the longest possible march: the box diagonal over delta, plus slack */
    double diag = 0.0;
    for (int a = 0; a < 3; ++a) diag += (g.hi[a] - g.lo[a]) * (g.hi[a] - g.lo[a]);
    int64_t cap = (int64_t)(sqrt(diag) / delta) + 4;
#pragma omp parallel
    {
        orc_sample *smp = (orc_sample *)malloc(sizeof(orc_sample) * (size_t)cap);
        double (*Rs)[3] = (double (*)[3])malloc(sizeof(double) * 3 * (size_t)cap);
#pragma omp for schedule(dynamic, 8)
        for (int64_t r = 0; r < n; ++r) {
            orc_ray_out res;
            double Y[ORC_NSH];
            orc_sh_basis(d + 3 * r, Y);
            int64_t ns = march(&g, o + 3 * r, d + 3 * r, delta, bg, stop, &res, smp, cap);
            if (ns > cap) ns = cap;
            if (ns == 0) continue;
            /* suffix sums R_s */
            for (int ch = 0; ch < 3; ++ch) Rs[ns - 1][ch] = res.T_end * bg[ch];
            for (int64_t s = ns - 2; s >= 0; --s)
                for (int ch = 0; ch < 3; ++ch)
                    Rs[s][ch] = Rs[s + 1][ch] + smp[s + 1].w * smp[s + 1].c[ch];
            const double *gr = grad_rgb + 3 * r;
            for (int64_t s = 0; s < ns; ++s) {
                const orc_sample *q = &smp[s];
                double T_next = q->T * (1.0 - q->alpha);
                double gsig = 0.0;
                if (q->sigma_pre > 0.0)
                    for (int ch = 0; ch < 3; ++ch) {
                        double term = gr[ch] * delta * (T_next * q->c[ch] - Rs[s][ch]);
                        if (abs_mode == 2)
                            gsig += fabs(gr[ch]) * delta * (T_next * fabs(q->c[ch]) + fabs(Rs[s][ch]));
                        else
                            gsig += abs_mode ? fabs(term) : term;
                    }
                double gk[ORC_NV - 1];
                for (int ch = 0; ch < 3; ++ch) {
                    double gc = gr[ch] * q->w;
                    double gpre = q->pre[ch] > 0.0 ? gc : 0.0;
                    for (int l = 0; l < ORC_NSH; ++l)
                        gk[ch * ORC_NSH + l] = abs_mode ? fabs(gpre * Y[l]) : gpre * Y[l];
                }
                for (int c = 0; c < 8; ++c) {
                    int32_t row = g.idx[q->node[c]];
                    if (row < 0) continue;
                    double w = q->cw[c];
                    double *dst = grad_rows + (int64_t)row * ORC_NV;
#pragma omp atomic
                    dst[0] += w * gsig;
                    for (int v = 0; v < ORC_NV - 1; ++v) {
#pragma omp atomic
                        dst[1 + v] += w * gk[v];
                    }
                }
            }
        }
        free(smp);
        free(Rs);
    }
}

void orc_render_backward(int64_t R, const int32_t *idx, const double *rows, int64_t row_stride,
                         const double *aabb, const double *o, const double *d, int64_t n,
                         const double *opts, const double *grad_rgb, double *grad_rows)
{
    render_backward_impl(R, idx, rows, row_stride, aabb, o, d, n, opts, grad_rgb, grad_rows, 0);
}

void orc_render_backward_abs(int64_t R, const int32_t *idx, const double *rows, int64_t row_stride,
                             const double *aabb, const double *o, const double *d, int64_t n,
                             const double *opts, const double *grad_rgb, double *grad_rows)
{
    render_backward_impl(R, idx, rows, row_stride, aabb, o, d, n, opts, grad_rgb, grad_rows, 1);
}

void orc_render_backward_mag(int64_t R, const int32_t *idx, const double *rows, int64_t row_stride,
                             const double *aabb, const double *o, const double *d, int64_t n,
                             const double *opts, const double *grad_rgb, double *grad_rows)
{
    render_backward_impl(R, idx, rows, row_stride, aabb, o, d, n, opts, grad_rgb, grad_rows, 2);
}

/* ------------------------------------------------------------------------- */
/* Maximum sample weight per node over a set of rays, the key of the        */
/* weight-threshold prune (Sec. 3.4 "Coarse to Fine": a voxel is dropped    */
/* when its weight T_i (1 - exp(-sigma_i delta_i)) stays under a threshold   */
/* on every training ray).  Samples and weights are those of orc_render.    */
/* Reading (values live on the nodes, Sec. 3): a sample counts toward every  */
/* one of the 8 corner nodes of the cell it lies in -- the nodes its values  */
/* are interpolated from -- whatever its trilinear weights; a NULL corner    */
/* has no row and takes nothing.                                             */
/*   wmax[row] = max(wmax[row], max over samples s crediting row of w_s)     */
/* wmax [M] is updated in place (callers start from zeros and may call again */
/* with more rays).                                                          */
/* ------------------------------------------------------------------------- */
void orc_max_weight(int64_t R, const int32_t *idx, const double *rows, int64_t row_stride,
                    const double *aabb, const double *o, const double *d, int64_t n,
                    const double *opts, double *wmax)
{
    orc_grid g;
    grid_init(&g, R, idx, rows, row_stride, aabb);
    double hmin = g.h[0] < g.h[1] ? g.h[0] : g.h[1];
    if (g.h[2] < hmin) hmin = g.h[2];
    double delta = opts[0] * hmin;
    double bg[3] = {opts[1], opts[2], opts[3]};
    double stop = opts[4];
    double diag = 0.0;
    for (int a = 0; a < 3; ++a) diag += (g.hi[a] - g.lo[a]) * (g.hi[a] - g.lo[a]);
    int64_t cap = (int64_t)(sqrt(diag) / delta) + 4;
#pragma omp parallel
    {
        orc_sample *smp = (orc_sample *)malloc(sizeof(orc_sample) * (size_t)cap);
#pragma omp for schedule(dynamic, 8)
        for (int64_t r = 0; r < n; ++r) {
            orc_ray_out res;
            int64_t ns = march(&g, o + 3 * r, d + 3 * r, delta, bg, stop, &res, smp, cap);
            if (ns > cap) ns = cap;
            for (int64_t s = 0; s < ns; ++s) {
                double w = smp[s].w;
                for (int c = 0; c < 8; ++c) {
                    int32_t row = g.idx[smp[s].node[c]];
                    if (row < 0) continue;
#pragma omp atomic compare
                    if (wmax[row] < w) { wmax[row] = w; }
                }
            }
        }
        free(smp);
    }
}

/* ------------------------------------------------------------------------- */
/* Cauchy sparsity prior on the samples' densities (Sec. 3.7, Eq. 4; the     */
/* paper uses it on real scenes, lambda_s 1e-12 / 1e-11 in Supp. B.3/B.4):   */
/*   L_s = lambda_s sum over rays r and samples k of log(1 + 2 sigma_rk^2)   */
/* over the samples each ray marches (those of orc_render, early stopping    */
/* included), sigma the activated density max(0, sigma_interp).  Adjoint:    */
/*   dL_s/dsigma_interp = lambda_s 4 sigma / (1 + 2 sigma^2), zero where     */
/*   sigma_interp <= 0,                                                      */
/* reaching each non-NULL corner with its trilinear weight.  Adds the        */
/* density column of grad_rows [M, 28] (FP64) and returns L_s.               */
/* ------------------------------------------------------------------------- */
double orc_sparsity(int64_t R, const int32_t *idx, const double *rows, int64_t row_stride,
                    const double *aabb, const double *o, const double *d, int64_t n,
                    const double *opts, double lambda_s, double *grad_rows)
{
    orc_grid g;
    grid_init(&g, R, idx, rows, row_stride, aabb);
    double hmin = g.h[0] < g.h[1] ? g.h[0] : g.h[1];
    if (g.h[2] < hmin) hmin = g.h[2];
    double delta = opts[0] * hmin;
    double bg[3] = {opts[1], opts[2], opts[3]};
    double stop = opts[4];
    double diag = 0.0;
    for (int a = 0; a < 3; ++a) diag += (g.hi[a] - g.lo[a]) * (g.hi[a] - g.lo[a]);
    int64_t cap = (int64_t)(sqrt(diag) / delta) + 4;
    double L = 0.0;
#pragma omp parallel reduction(+ : L)
    {
        orc_sample *smp = (orc_sample *)malloc(sizeof(orc_sample) * (size_t)cap);
#pragma omp for schedule(dynamic, 8)
        for (int64_t r = 0; r < n; ++r) {
            orc_ray_out res;
            int64_t ns = march(&g, o + 3 * r, d + 3 * r, delta, bg, stop, &res, smp, cap);
            if (ns > cap) ns = cap;
            for (int64_t s = 0; s < ns; ++s) {
                double sig = smp[s].sigma;
                L += log(1.0 + 2.0 * sig * sig);
                if (!grad_rows || !(smp[s].sigma_pre > 0.0)) continue;
                double gs = lambda_s * 4.0 * sig / (1.0 + 2.0 * sig * sig);
                for (int c = 0; c < 8; ++c) {
                    int32_t row = g.idx[smp[s].node[c]];
                    if (row < 0) continue;
#pragma omp atomic
                    grad_rows[(int64_t)row * ORC_NV] += smp[s].cw[c] * gs;
                }
            }
        }
        free(smp);
    }
    return lambda_s * L;
}

/* ------------------------------------------------------------------------- */
/* MSE reconstruction loss over the ray batch (Eq. 3, Sec. 3.5):             */
/*   L = 1/|R| sum_r ||C_r - Chat_r||_2^2,  dL/dChat = 2 (Chat - C) / |R|.   */
/* ------------------------------------------------------------------------- */
double orc_mse(const double *pred, const double *target, int64_t n, double *grad)
{
    double L = 0.0;
    for (int64_t r = 0; r < n; ++r)
        for (int ch = 0; ch < 3; ++ch) {
            double e = pred[3 * r + ch] - target[3 * r + ch];
            L += e * e;
            if (grad) grad[3 * r + ch] = 2.0 * e / (double)n;
        }
    return L / (double)n;
}

/* ------------------------------------------------------------------------- */
/* Total variation (Sec. 3.5 loss; Supp. B.1 normalisation and edge rules).  */
/* For each selected node v and value d:                                     */
/*   D_a(v,d) = (V_d(v + e_a) - V_d(v)) * R / 256                            */
/*   t(v,d)   = sqrt(D_x^2 + D_y^2 + D_z^2)                                  */
/* L_TV = sum_{v in S} sum_d lambda_d / |S| * t(v,d), lambda_0 = lambda_sigma*/
/* and lambda_{d>0} = lambda_sh.  A missing neighbour (NULL or outside the   */
/* grid) has value 0 for density and V_d(v) for SH.  Gradients reach only    */
/* occupied rows; t = 0 gives zero gradient.  Selection = segments of        */
/* consecutive linear node ids.  Returns the loss; grad_rows [M,28] (+=).    */
/* ------------------------------------------------------------------------- */
double orc_tv(int64_t R, const int32_t *idx, const double *rows, int64_t row_stride,
              const int64_t *seg_start, const int64_t *seg_len, int64_t n_seg,
              double lambda_sigma, double lambda_sh, double *grad_rows)
{
    orc_grid g;
    double aabb[6] = {-1, -1, -1, 1, 1, 1};
    grid_init(&g, R, idx, rows, row_stride, aabb);
    int64_t n_sel = 0;
    for (int64_t q = 0; q < n_seg; ++q) n_sel += seg_len[q];
    if (n_sel == 0) return 0.0;
    double scale = (double)R / 256.0;
    double L = 0.0;
    for (int64_t q = 0; q < n_seg; ++q) {
        for (int64_t n = seg_start[q]; n < seg_start[q] + seg_len[q]; ++n) {
            int64_t i = n / (R * R), j = (n / R) % R, k = n % R;
            int64_t nb[3];
            nb[0] = i + 1 < R ? node_id(R, i + 1, j, k) : -1;
            nb[1] = j + 1 < R ? node_id(R, i, j + 1, k) : -1;
            nb[2] = k + 1 < R ? node_id(R, i, j, k + 1) : -1;
            int32_t self_row = idx[n];
            for (int d = 0; d < ORC_NV; ++d) {
                double lam = (d == 0 ? lambda_sigma : lambda_sh) / (double)n_sel;
                double self = node_value(&g, n, d);
                double D[3];
                int nb_present[3];
                for (int a = 0; a < 3; ++a) {
                    nb_present[a] = nb[a] >= 0 && idx[nb[a]] >= 0;
                    double nv;
                    if (nb_present[a]) nv = node_value(&g, nb[a], d);
                    else nv = (d == 0) ? 0.0 : self;
                    D[a] = (nv - self) * scale;
                }
                double t = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
                L += lam * t;
                if (t == 0.0 || !grad_rows) continue;
                for (int a = 0; a < 3; ++a) {
                    /* dD_a/dV(neighbour) = scale when the neighbour is present */
                    if (nb_present[a])
                        grad_rows[(int64_t)idx[nb[a]] * ORC_NV + d] += lam * D[a] * scale / t;
                }
                if (self_row >= 0) {
                    double gs = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        /* dD_a/dV(v) = -scale, except for a missing SH neighbour,
                         * where D_a = V(v) - V(v) does not depend on V(v). */
                        if (nb_present[a] || d == 0) gs += -scale * D[a] / t;
                    }
                    grad_rows[(int64_t)self_row * ORC_NV + d] += lam * gs;
                }
            }
        }
    }
    return L;
}

/* ------------------------------------------------------------------------- */
/* RMSProp (Sec. 3.5), applied to every entry with a non-zero gradient:      */
/*   v <- beta v + (1 - beta) g^2 ;  x <- x - lr g / (sqrt(v) + eps) ; g <- 0 */
/* lr = lr_sigma for column 0 (density) and lr_sh for the SH columns.        */
/* x, v, grad are [M, 28] FP64.                                              */
/* ------------------------------------------------------------------------- */
void orc_rmsprop(int64_t M, double *x, double *v, double *grad, double lr_sigma, double lr_sh,
                 double beta, double eps)
{
    for (int64_t m = 0; m < M; ++m)
        for (int d = 0; d < ORC_NV; ++d) {
            int64_t e = m * ORC_NV + d;
            double gg = grad[e];
            if (gg == 0.0) continue;
            double lr = d == 0 ? lr_sigma : lr_sh;
            v[e] = beta * v[e] + (1.0 - beta) * gg * gg;
            x[e] = x[e] - lr * gg / (sqrt(v[e]) + eps);
            grad[e] = 0.0;
        }
}

/* ------------------------------------------------------------------------- */
/* Pruning with dilation (Sec. 3.4 "Coarse to Fine").  A node is hot when it */
/* is occupied and its key is at least tau; the key is its density (the     */
/* density-threshold form) or a per-row value the caller supplies (the       */
/* weight-threshold form, with the rows' maximum weights, orc_max_weight).   */
/* hot(n)  = node n occupied and key(n) >= tau                               */
/* keep(n) = node n occupied and (dilate ? any hot node in the 3x3x3         */
/*           neighbourhood of n clipped to the grid : hot(n))                */
/* Kept nodes get new row ids in ascending n; their rows are copied.         */
/* idx_out [R^3]; rows_out [n_keep, row_stride] may be NULL (count only).    */
/* Returns n_keep.                                                           */
/* ------------------------------------------------------------------------- */
static int64_t prune_impl(int64_t R, const int32_t *idx, const double *rows, int64_t row_stride,
                          const double *key, double tau, int dilate, int32_t *idx_out, double *rows_out)
{
    int64_t N = R * R * R;
    unsigned char *hot = (unsigned char *)malloc((size_t)N);
    for (int64_t n = 0; n < N; ++n) {
        hot[n] = 0;
        if (idx[n] < 0) continue;
        double k = key ? key[idx[n]] : rows[(int64_t)idx[n] * row_stride];
        hot[n] = k >= tau;
    }
    int64_t next = 0;
    for (int64_t n = 0; n < N; ++n) {
        int keep = 0;
        if (idx[n] >= 0) {
            if (!dilate) {
                keep = hot[n];
            } else {
                int64_t i = n / (R * R), j = (n / R) % R, k = n % R;
                for (int64_t di = -1; di <= 1 && !keep; ++di)
                    for (int64_t dj = -1; dj <= 1 && !keep; ++dj)
                        for (int64_t dk = -1; dk <= 1 && !keep; ++dk) {
                            int64_t a = i + di, b = j + dj, c = k + dk;
                            if (a < 0 || b < 0 || c < 0 || a >= R || b >= R || c >= R) continue;
                            if (hot[node_id(R, a, b, c)]) keep = 1;
                        }
            }
        }
        if (keep) {
            if (idx_out) idx_out[n] = (int32_t)next;
            if (rows_out)
                memcpy(rows_out + next * row_stride, rows + (int64_t)idx[n] * row_stride,
                       sizeof(double) * (size_t)row_stride);
            ++next;
        } else if (idx_out) {
            idx_out[n] = -1;
        }
    }
    free(hot);
    return next;
}

/* density-threshold form: key = sigma (row column 0) */
int64_t orc_prune(int64_t R, const int32_t *idx, const double *rows, int64_t row_stride,
                  double tau, int dilate, int32_t *idx_out, double *rows_out)
{
    return prune_impl(R, idx, rows, row_stride, NULL, tau, dilate, idx_out, rows_out);
}

/* weight-threshold form: key [M], one value per row */
int64_t orc_prune_key(int64_t R, const int32_t *idx, const double *rows, int64_t row_stride,
                      const double *key, double tau, int dilate, int32_t *idx_out, double *rows_out)
{
    return prune_impl(R, idx, rows, row_stride, key, tau, dilate, idx_out, rows_out);
}

/* ------------------------------------------------------------------------- */
/* Upsample R -> R2 by trilinear interpolation (Sec. 3.4 "Coarse to Fine":   */
/* subdivide, initialise by trilinear interpolation; any resolution).       */
/* New node i' along an axis sits at old grid coordinate i'(R-1)/(R2-1):     */
/*   base = floor(i'(R-1)/(R2-1)) (integer division), rem = i'(R-1) mod (R2-1)*/
/*   frac = rem / (R2-1); the +1 corner has weight frac and exists only when  */
/*   rem != 0.  A new node is occupied iff one of its support nodes (corners  */
/*   with non-zero weight) is occupied; values interpolate with NULL = 0.    */
/* Occupied new nodes get row ids in ascending n'.  rows_out [M', 28] FP64  */
/* (may be NULL for a count).  Returns M'.                                   */
/* ------------------------------------------------------------------------- */
int64_t orc_upsample(int64_t R, const int32_t *idx, const double *rows, int64_t row_stride,
                     int64_t R2, int32_t *idx_out, double *rows_out)
{
    orc_grid g;
    double aabb[6] = {-1, -1, -1, 1, 1, 1};
    grid_init(&g, R, idx, rows, row_stride, aabb);
    int64_t next = 0;
    for (int64_t i2 = 0; i2 < R2; ++i2)
        for (int64_t j2 = 0; j2 < R2; ++j2)
            for (int64_t k2 = 0; k2 < R2; ++k2) {
                int64_t p[3] = {i2, j2, k2};
                int64_t base[3], rem[3];
                double f[3];
                for (int a = 0; a < 3; ++a) {
                    int64_t num = p[a] * (R - 1);
                    base[a] = num / (R2 - 1);
                    rem[a] = num % (R2 - 1);
                    f[a] = (double)rem[a] / (double)(R2 - 1);
                }
                int occ = 0;
                double val[ORC_NV];
                for (int d = 0; d < ORC_NV; ++d) val[d] = 0.0;
                for (int c = 0; c < 8; ++c) {
                    int cb[3] = {(c >> 2) & 1, (c >> 1) & 1, c & 1};
                    int support = 1;
                    double w = 1.0;
                    for (int a = 0; a < 3; ++a) {
                        if (cb[a] && rem[a] == 0) support = 0;
                        w *= cb[a] ? f[a] : 1.0 - f[a];
                    }
                    if (!support) continue;
                    int64_t n = node_id(R, base[0] + cb[0], base[1] + cb[1], base[2] + cb[2]);
                    if (idx[n] >= 0) occ = 1;
                    for (int d = 0; d < ORC_NV; ++d) val[d] += w * node_value(&g, n, d);
                }
                int64_t n2 = node_id(R2, i2, j2, k2);
                if (occ) {
                    if (idx_out) idx_out[n2] = (int32_t)next;
                    if (rows_out)
                        for (int d = 0; d < ORC_NV; ++d) rows_out[next * ORC_NV + d] = val[d];
                    ++next;
                } else if (idx_out) {
                    idx_out[n2] = -1;
                }
            }
    return next;
}

/* ------------------------------------------------------------------------- */
/* FP32 -> BF16 storage rounding, round-to-nearest-even, for the oracle of   */
/* the BF16-SH storage form: values are rounded, then used exactly in FP64.  */
/* In place on n floats; finite inputs only.                                 */
/* ------------------------------------------------------------------------- */
void orc_round_bf16(float *x, int64_t n)
{
    for (int64_t q = 0; q < n; ++q) {
        uint32_t u;
        memcpy(&u, &x[q], 4);
        uint32_t lower = u & 0xFFFFu;
        uint32_t upper = u >> 16;
        if (lower > 0x8000u || (lower == 0x8000u && (upper & 1u))) upper += 1u;
        u = upper << 16;
        memcpy(&x[q], &u, 4);
    }
}

/* Number of threads the OpenMP regions use (1 without OpenMP). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sets the number of threads later OpenMP regions use (no effect without OpenMP). */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

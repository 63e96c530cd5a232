/*
 * vr_oracle.c -- plain, slow, FP64 CPU oracle for the data-parallel volume
 * rendering path (per-brick emission-absorption ray marching + sort-last
 * "over" compositing).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do. It shares no code, header or table with the CUDA
 * path.
 *
 * What the paper fixes and what it does not:
 *   - Sec. 2.2: the data is spatially distributed over ranks ("each rank gets
 *     a share"), possibly unevenly; each rank renders what it holds.
 *   - Sec. 3: the frame's image ends up in one framebuffer on the main rank
 *     (DP-ANARI conventions); Sec. 4: processes "render and composite images"
 *     headless, several data parts per GPU.
 *   - The paper gives no rendering formula. Every formula below is the
 *     standard emission-absorption optical model (Max 1995, "Optical Models
 *     for Direct Volume Rendering") discretised as a front-to-back Riemann
 *     sum, with the readings written out at each function.
 *
 * Everything is evaluated in double precision; stored f32/bf16/f16 values
 * are converted to double exactly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- input descriptions (mirrored field-for-field by oracle/__init__.py) -- */

typedef struct {
    int ortho;
    double eye[3], dir[3], up[3];
    double fovy_deg, ortho_w, ortho_h;
    int width, height;
} orc_camera;

enum { ORC_F32 = 0, ORC_BF16 = 1, ORC_F16 = 2, ORC_F64 = 3 };

typedef struct {
    const void *vol;        /* x fastest, [Nz][Ny][Nx] */
    int dtype;              /* ORC_* */
    int dims[3];            /* Nx, Ny, Nz */
    int nb;                 /* number of bricks */
    const int *boxes;       /* nb x 6: lo x,y,z then hi x,y,z (half-open voxel box) */
    const float *tf;        /* ntf x 4 RGBA */
    int ntf;
    double vmin, vmax;      /* classification range (global, never per brick) */
    orc_camera cam;
    double step_voxels;     /* sample spacing in voxel widths */
    double ert_alpha;       /* early termination opacity; >= 1 disables */
    double ert_bias;        /* added to the termination threshold (ambiguity probes) */
    double end_bias;        /* added to t_out in the sample-count test (ambiguity probes) */
} orc_scene;

/* ---- scalar helpers ---------------------------------------------------- */

static double half_to_double(uint16_t h)
{
    int s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0)
        v = ldexp((double)m, -24);
    else if (e == 31)
        v = m ? NAN : INFINITY;
    else
        v = ldexp((double)(1024 + m), e - 25);
    return s ? -v : v;
}

static double bf16_to_double(uint16_t b)
{
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double voxel(const orc_scene *sc, long long idx)
{
    switch (sc->dtype) {
    case ORC_F32: return (double)((const float *)sc->vol)[idx];
    case ORC_BF16: return bf16_to_double(((const uint16_t *)sc->vol)[idx]);
    case ORC_F16: return half_to_double(((const uint16_t *)sc->vol)[idx]);
    default: return ((const double *)sc->vol)[idx];
    }
}

static int clampi(long long v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : (int)v); }
static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

static int nmax3(const int d[3])
{
    int m = d[0] > d[1] ? d[0] : d[1];
    return m > d[2] ? m : d[2];
}

/* ---- sampling: trilinear reconstruction, clamp-to-edge ----------------
 * Reading (paper silent): the volume occupies [0,Nx/Nmax]x[0,Ny/Nmax]x
 * [0,Nz/Nmax]; voxel (i,j,k) sits at its cell centre ((i+.5)/Nmax, ...).
 * Per axis v = p*Nmax - 0.5, i0 = floor(v), f = v - i0; the two indices are
 * clamped to [0, N-1]; the value is the 8-corner tensor-product blend. */
static double sample_trilinear(const orc_scene *sc, const double p[3])
{
    const int nm = nmax3(sc->dims);
    int i0[3], i1[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double v = p[a] * nm - 0.5;
        double fl = floor(v);
        f[a] = v - fl;
        i0[a] = clampi((long long)fl, 0, sc->dims[a] - 1);
        i1[a] = clampi((long long)fl + 1, 0, sc->dims[a] - 1);
    }
    const long long nx = sc->dims[0], nxy = (long long)sc->dims[0] * sc->dims[1];
    double s = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) *
                           (dz ? f[2] : 1.0 - f[2]);
                long long idx = (dz ? i1[2] : i0[2]) * nxy + (dy ? i1[1] : i0[1]) * nx +
                                (dx ? i1[0] : i0[0]);
                s += w * voxel(sc, idx);
            }
    return s;
}

/* ---- classification: 1D RGBA transfer function ------------------------
 * Reading (paper silent): u = clamp((s - vmin)/(vmax - vmin), 0, 1) with the
 * global range; entry i of n sits at u = i/(n-1); x = u(n-1),
 * i = min(floor(x), n-2), w = x - i, rgba = (1-w) T[i] + w T[i+1]. The alpha is
 * the opacity of one sample at the configured step (no step correction). */
static void classify(const orc_scene *sc, double s, double rgba[4])
{
    double u = clampd((s - sc->vmin) / (sc->vmax - sc->vmin), 0.0, 1.0);
    double x = u * (sc->ntf - 1);
    int i = (int)floor(x);
    if (i > sc->ntf - 2) i = sc->ntf - 2;
    double w = x - i;
    for (int c = 0; c < 4; ++c)
        rgba[c] = (1.0 - w) * (double)sc->tf[4 * i + c] + w * (double)sc->tf[4 * (i + 1) + c];
}

/* ---- primary rays (Sec. 2.1: rays originate at the virtual camera) -----
 * Basis: f = dir/|dir|, r = (up x f)/|up x f|, u = f x r.
 * Orthographic: origin = eye + ((px+.5)/W - .5) w r + ((py+.5)/H - .5) h u,
 *   direction f.
 * Perspective: origin = eye, direction = normalise(f + sx r + sy u) with
 *   sy = ((py+.5)/H*2 - 1) tan(fovy/2), sx = ((px+.5)/W*2 - 1) tan(fovy/2) W/H. */
static void norm3(double v[3])
{
    double l = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= l; v[1] /= l; v[2] /= l;
}

static void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static void primary_ray(const orc_camera *cam, int px, int py, double o[3], double d[3])
{
    double f[3] = {cam->dir[0], cam->dir[1], cam->dir[2]}, r[3], u[3];
    norm3(f);
    cross3(cam->up, f, r);
    norm3(r);
    cross3(f, r, u);
    double fx = (px + 0.5) / cam->width, fy = (py + 0.5) / cam->height;
    if (cam->ortho) {
        double a = (fx - 0.5) * cam->ortho_w, b = (fy - 0.5) * cam->ortho_h;
        for (int i = 0; i < 3; ++i) {
            o[i] = cam->eye[i] + a * r[i] + b * u[i];
            d[i] = f[i];
        }
    } else {
        double th = tan(cam->fovy_deg * M_PI / 360.0);
        double sx = (fx * 2.0 - 1.0) * th * ((double)cam->width / cam->height);
        double sy = (fy * 2.0 - 1.0) * th;
        for (int i = 0; i < 3; ++i) {
            o[i] = cam->eye[i];
            d[i] = f[i] + sx * r[i] + sy * u[i];
        }
        norm3(d);
    }
}

/* Slab test against the whole-volume box [0,E]; returns 0 on a miss.
 * Reading: t_in = max(t_near, 0), the ray enters at t_in and leaves at t_out;
 * an axis with d = 0 constrains nothing if the origin lies within the slab. */
static int volume_interval(const double E[3], const double o[3], const double d[3],
                           double *t_in, double *t_out)
{
    double t0 = -INFINITY, t1 = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < 0.0 || o[a] > E[a]) return 0;
            continue;
        }
        double ta = (0.0 - o[a]) / d[a], tb = (E[a] - o[a]) / d[a];
        double tn = ta < tb ? ta : tb, tf = ta < tb ? tb : ta;
        if (tn > t0) t0 = tn;
        if (tf < t1) t1 = tf;
    }
    if (t0 < 0.0) t0 = 0.0;
    if (!(t0 < t1)) return 0;
    *t_in = t0;
    *t_out = t1;
    return 1;
}

static int in_box(const int *box, const int c[3])
{
    return c[0] >= box[0] && c[0] < box[3] && c[1] >= box[1] && c[1] < box[4] &&
           c[2] >= box[2] && c[2] < box[5];
}

/* ---- one pixel ----------------------------------------------------------
 * Global lattice (reading; brick-independent): t_k = t_in + (k + 1/2) dt for
 * k = 0, 1, ... while t_k < t_out, dt = step_voxels / Nmax in world units.
 * Ownership: sample k at p = o + t_k d belongs to the brick whose half-open
 * voxel box contains the cell clamp(floor(p Nmax), 0, N-1) (Sec. 2.2: each rank
 * renders exactly its share of the data; the shares tile the domain).
 * Each brick accumulates its own samples front to back from C = 0, T = 1:
 * C += T alpha rgb, T *= (1 - alpha); its partial is (C, 1 - T), rgb
 * premultiplied. Early termination (reading): after a sample, the brick stops if
 * T <= 1 - ert_alpha (+ ert_bias). The pixel is the front-to-back "over"
 * (Sec. 3/4: the per-rank images are composited) of the partials in the order
 * the ray meets the bricks: C <- C + (1-A) C_b, A <- A + (1-A) A_b. */
typedef struct {
    double *C;      /* nb x 3 */
    double *T;      /* nb */
    long long *first; /* nb: index of the first owned sample, -1 if none */
    char *done;     /* nb */
    int *order;     /* nb */
    int bad;        /* set when a sample's cell lies in no brick */
} pixel_ws;

static long long render_pixel(const orc_scene *sc, int px, int py, pixel_ws *ws,
                              double out[4], double *partials_px, long long pstride)
{
    const int nb = sc->nb;
    const int nm = nmax3(sc->dims);
    const double E[3] = {(double)sc->dims[0] / nm, (double)sc->dims[1] / nm,
                         (double)sc->dims[2] / nm};
    for (int b = 0; b < nb; ++b) {
        ws->C[3 * b] = ws->C[3 * b + 1] = ws->C[3 * b + 2] = 0.0;
        ws->T[b] = 1.0;
        ws->first[b] = -1;
        ws->done[b] = 0;
    }
    out[0] = out[1] = out[2] = out[3] = 0.0;
    long long executed = 0;
    double o[3], d[3], t_in, t_out;
    primary_ray(&sc->cam, px, py, o, d);
    if (volume_interval(E, o, d, &t_in, &t_out)) {
        const double dt = sc->step_voxels / nm;
        const int ert = sc->ert_alpha < 1.0;
        const double thr = (1.0 - sc->ert_alpha) + sc->ert_bias;
        int cur = 0;
        for (long long k = 0;; ++k) {
            double t = t_in + (k + 0.5) * dt;
            if (!(t < t_out + sc->end_bias)) break;
            double p[3];
            int c[3];
            for (int a = 0; a < 3; ++a) {
                p[a] = o[a] + t * d[a];
                c[a] = clampi((long long)floor(p[a] * nm), 0, sc->dims[a] - 1);
            }
            if (!in_box(sc->boxes + 6 * cur, c)) {
                cur = -1;
                for (int b = 0; b < nb; ++b)
                    if (in_box(sc->boxes + 6 * b, c)) { cur = b; break; }
                if (cur < 0) { cur = 0; ws->bad = 1; continue; } /* partition leaves a gap */
            }
            if (ws->first[cur] < 0) ws->first[cur] = k;
            if (ws->done[cur]) continue;
            double rgba[4];
            classify(sc, sample_trilinear(sc, p), rgba);
            double Tb = ws->T[cur];
            for (int ch = 0; ch < 3; ++ch) ws->C[3 * cur + ch] += Tb * rgba[3] * rgba[ch];
            ws->T[cur] = Tb * (1.0 - rgba[3]);
            ++executed;
            if (ert && ws->T[cur] <= thr) ws->done[cur] = 1;
        }
        /* front-to-back order along this ray = order of first owned sample */
        int m = 0;
        for (int b = 0; b < nb; ++b)
            if (ws->first[b] >= 0) {
                int j = m++;
                while (j > 0 && ws->first[ws->order[j - 1]] > ws->first[b]) {
                    ws->order[j] = ws->order[j - 1];
                    --j;
                }
                ws->order[j] = b;
            }
        for (int j = 0; j < m; ++j) {
            int b = ws->order[j];
            double Ab = 1.0 - ws->T[b], w = 1.0 - out[3];
            for (int ch = 0; ch < 3; ++ch) out[ch] += w * ws->C[3 * b + ch];
            out[3] += w * Ab;
        }
    }
    if (partials_px)
        for (int b = 0; b < nb; ++b) {
            double *q = partials_px + b * pstride;
            int vis = ws->first[b] >= 0;
            q[0] = vis ? ws->C[3 * b] : 0.0;
            q[1] = vis ? ws->C[3 * b + 1] : 0.0;
            q[2] = vis ? ws->C[3 * b + 2] : 0.0;
            q[3] = vis ? 1.0 - ws->T[b] : 0.0;
        }
    return executed;
}

/* Render a list of pixels (m x 2 ints: px, py).
 *   img      m x 4 composited RGBA (premultiplied rgb, alpha = 1 - T)
 *   partials nb x m x 4 per-brick partials (may be NULL)
 *   nsamples executed sample count over the list (may be NULL)
 * Returns 0 on success, -1 on allocation failure, -2 on bad arguments, -4 if
 * a sample fell in a cell that no brick covers (the boxes do not tile). */
int orc_render_pixels(const orc_scene *sc, int m, const int *pix, double *img,
                      double *partials, long long *nsamples, int nthreads)
{
    if (!sc || sc->nb < 1 || sc->ntf < 2 || !(sc->vmax > sc->vmin) || sc->step_voxels <= 0)
        return -2;
    long long total = 0;
    int fail = 0;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads) reduction(+ : total) reduction(| : fail)
    {
        pixel_ws ws;
        const int nb = sc->nb;
        ws.C = (double *)malloc(sizeof(double) * 3 * nb);
        ws.T = (double *)malloc(sizeof(double) * nb);
        ws.first = (long long *)malloc(sizeof(long long) * nb);
        ws.done = (char *)malloc(nb);
        ws.order = (int *)malloc(sizeof(int) * nb);
        ws.bad = 0;
        if (!ws.C || !ws.T || !ws.first || !ws.done || !ws.order) {
            fail = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int i = 0; i < m; ++i)
                total += render_pixel(sc, pix[2 * i], pix[2 * i + 1], &ws, img + 4 * (long long)i,
                                      partials ? partials + 4 * (long long)i : NULL,
                                      4 * (long long)m);
            if (ws.bad) fail |= 2;
        }
        free(ws.C); free(ws.T); free(ws.first); free(ws.done); free(ws.order);
    }
    if (nsamples) *nsamples = total;
    if (fail & 1) return -1;
    return (fail & 2) ? -4 : 0;
}

/* ---- partitions (Sec. 2.2 spatial distribution; Sec. 4 uneven shares) ----
 * Regular grid: boundaries floor(N j / g), j = 0..g, per axis; brick id
 * (bz gy + by) gx + bx. */
int orc_grid_partition(const int dims[3], const int g[3], int *boxes)
{
    for (int a = 0; a < 3; ++a)
        if (g[a] < 1 || g[a] > dims[a]) return -2;
    int id = 0;
    for (int bz = 0; bz < g[2]; ++bz)
        for (int by = 0; by < g[1]; ++by)
            for (int bx = 0; bx < g[0]; ++bx, ++id) {
                int b[3] = {bx, by, bz};
                for (int a = 0; a < 3; ++a) {
                    boxes[6 * id + a] = (int)(((long long)dims[a] * b[a]) / g[a]);
                    boxes[6 * id + 3 + a] = (int)(((long long)dims[a] * (b[a] + 1)) / g[a]);
                }
            }
    return 0;
}

/* kd partition (reading; the paper only notes uneven distributions, Sec. 4):
 * until n leaves exist, take the leaf with the most voxels (ties: lowest id),
 * cut it across its longest axis (ties: x before y before z) at
 * lo + round(u_j * extent), clamped so both halves are non-empty, with u_j the
 * j-th given fraction. The low half keeps the leaf's id, the high half becomes
 * leaf number (current count). */
int orc_kd_partition(const int dims[3], int n, const double *u, int *boxes)
{
    if (n < 1) return -2;
    boxes[0] = boxes[1] = boxes[2] = 0;
    boxes[3] = dims[0]; boxes[4] = dims[1]; boxes[5] = dims[2];
    for (int count = 1; count < n; ++count) {
        int best = -1;
        long long bestv = -1;
        for (int l = 0; l < count; ++l) {
            const int *b = boxes + 6 * l;
            long long v = (long long)(b[3] - b[0]) * (b[4] - b[1]) * (b[5] - b[2]);
            if (v > bestv) { bestv = v; best = l; }
        }
        int *b = boxes + 6 * best;
        int axis = 0;
        for (int a = 1; a < 3; ++a)
            if (b[3 + a] - b[a] > b[3 + axis] - b[axis]) axis = a;
        int ext = b[3 + axis] - b[axis];
        if (ext < 2) return -3; /* cannot split further */
        int cut = b[axis] + (int)floor(u[count - 1] * ext + 0.5);
        if (cut < b[axis] + 1) cut = b[axis] + 1;
        if (cut > b[3 + axis] - 1) cut = b[3 + axis] - 1;
        int *nbx = boxes + 6 * count;
        memcpy(nbx, b, 6 * sizeof(int));
        b[3 + axis] = cut;
        nbx[axis] = cut;
    }
    return 0;
}

/* Point probes of the two per-sample stages, for function-level pins. */
double orc_sample(const orc_scene *sc, const double p[3]) { return sample_trilinear(sc, p); }
void orc_classify(const orc_scene *sc, double s, double rgba[4]) { classify(sc, s, rgba); }
void orc_primary_ray(const orc_camera *cam, int px, int py, double o[3], double d[3])
{
    primary_ray(cam, px, py, o, d);
}

int orc_version(void) { return 1; }

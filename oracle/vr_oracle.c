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
    const double *tf64;     /* optional: ntf x 4 table in double, used instead of tf */
    int ert_global;         /* ray-state cycling: one (C, T) along the whole ray, global termination */
    double opc_ratio;       /* opacity correction step/reference step; 0 or 1 = off */
    /* tetrahedral mesh (unstructured elements). When mesh_tets is set the
     * samples come from the mesh and vol/dtype are unused; dims still fix the
     * domain box, the lattice spacing and the ownership cells. */
    const double *mesh_verts; /* nv x 3 world positions */
    const double *mesh_vals;  /* nv vertex values */
    const int *mesh_tets;     /* nt x 4 vertex indices */
    long long mesh_nt;
    int mesh_nv;
    int mesh_bruteforce;      /* 1: search every element of the brick (no bins) */
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

/* ---- sampling: tetrahedral mesh (unstructured elements) ----------------
 * The paper's data set is a mixed finite-element mesh distributed over ranks
 * (Sec. 5); here elements are tetrahedra, each held by one brick (rank).
 * Readings (the paper is silent on the sampling rule):
 *   - element e belongs to the brick whose box contains its centroid's cell
 *     clamp(floor(centroid Nmax), 0, N-1);
 *   - a lattice sample keeps the owner of Sec. 2.2's reading (its cell's
 *     brick) and takes its value from the owner's elements: the linear
 *     interpolant sum_i lambda_i s_i of the element that maximises
 *     min_i lambda_i(p), the barycentric coordinates of p. For p inside an
 *     element that is the element; on a shared face every candidate gives the
 *     same value (the interpolant is continuous on a conforming mesh); p
 *     outside every element by rounding, or outside the domain box, takes the
 *     nearest one.
 * Barycentrics by Cramer's rule on the edge matrix [v1-v0, v2-v0, v3-v0]. */
static void cross3(const double a[3], const double b[3], double o[3]);

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static double det3(const double a[3], const double b[3], const double c[3])
{
    double bc[3];
    cross3(b, c, bc);
    return dot3(a, bc);
}

static double tet_bary(const orc_scene *sc, long long e, const double p[3], double lam[4])
{
    const int *t = sc->mesh_tets + 4 * e;
    const double *v0 = sc->mesh_verts + 3 * (long long)t[0];
    double a[3], b[3], c[3], r[3];
    for (int i = 0; i < 3; ++i) {
        a[i] = sc->mesh_verts[3 * (long long)t[1] + i] - v0[i];
        b[i] = sc->mesh_verts[3 * (long long)t[2] + i] - v0[i];
        c[i] = sc->mesh_verts[3 * (long long)t[3] + i] - v0[i];
        r[i] = p[i] - v0[i];
    }
    const double det = det3(a, b, c);
    lam[1] = det3(r, b, c) / det;
    lam[2] = det3(a, r, c) / det;
    lam[3] = det3(a, b, r) / det;
    lam[0] = 1.0 - lam[1] - lam[2] - lam[3];
    double m = lam[0];
    for (int i = 1; i < 4; ++i)
        if (lam[i] < m) m = lam[i];
    return m;
}

/* Element lists: by brick, and by a uniform grid of bins over the domain box
 * (each element in every bin its bounding box, widened by 1e-9, overlaps). The
 * bins only narrow the candidates: an element whose closed box misses p has a
 * negative coordinate at p and cannot beat the element containing p. */
typedef struct {
    int *brick;          /* nt */
    long long *bstart;   /* nb + 1 */
    int *bitems;
    int r[3];
    double E[3];
    long long *start;    /* bins + 1 */
    int *items;
} mesh_index;

static void mesh_index_free(mesh_index *mi)
{
    free(mi->brick); free(mi->bstart); free(mi->bitems); free(mi->start); free(mi->items);
    memset(mi, 0, sizeof(*mi));
}

static int in_box(const int *box, const int c[3]);

static int mesh_bin(const mesh_index *mi, int a, double x)
{
    return clampi((long long)floor(x / mi->E[a] * mi->r[a]), 0, mi->r[a] - 1);
}

/* Returns 0, -1 on allocation failure, -2 on a bad element index. */
static int mesh_index_build(const orc_scene *sc, mesh_index *mi)
{
    memset(mi, 0, sizeof(*mi));
    const long long nt = sc->mesh_nt;
    const int nb = sc->nb, nm = nmax3(sc->dims);
    for (long long e = 0; e < 4 * nt; ++e)
        if (sc->mesh_tets[e] < 0 || sc->mesh_tets[e] >= sc->mesh_nv) return -2;
    mi->brick = (int *)malloc(sizeof(int) * (nt > 0 ? nt : 1));
    mi->bstart = (long long *)calloc(nb + 1, sizeof(long long));
    mi->bitems = (int *)malloc(sizeof(int) * (nt > 0 ? nt : 1));
    if (!mi->brick || !mi->bstart || !mi->bitems) { mesh_index_free(mi); return -1; }
    for (long long e = 0; e < nt; ++e) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            double m = 0.0;
            for (int j = 0; j < 4; ++j) m += sc->mesh_verts[3 * (long long)sc->mesh_tets[4 * e + j] + a];
            c[a] = clampi((long long)floor(m / 4.0 * nm), 0, sc->dims[a] - 1);
        }
        mi->brick[e] = -1;
        for (int b = 0; b < nb; ++b)
            if (in_box(sc->boxes + 6 * b, c)) { mi->brick[e] = b; break; }
        if (mi->brick[e] >= 0) mi->bstart[mi->brick[e] + 1]++;
    }
    for (int b = 0; b < nb; ++b) mi->bstart[b + 1] += mi->bstart[b];
    {
        long long *fill = (long long *)malloc(sizeof(long long) * (nb + 1));
        if (!fill) { mesh_index_free(mi); return -1; }
        memcpy(fill, mi->bstart, sizeof(long long) * (nb + 1));
        for (long long e = 0; e < nt; ++e)
            if (mi->brick[e] >= 0) mi->bitems[fill[mi->brick[e]]++] = (int)e;
        free(fill);
    }
    double side = cbrt((double)(nt > 2 ? nt : 2) / 2.0);
    for (int a = 0; a < 3; ++a) {
        mi->E[a] = (double)sc->dims[a] / nm;
        int r = (int)ceil(side * mi->E[a]);
        mi->r[a] = r < 1 ? 1 : (r > 128 ? 128 : r);
    }
    const long long nbins = (long long)mi->r[0] * mi->r[1] * mi->r[2];
    mi->start = (long long *)calloc(nbins + 1, sizeof(long long));
    if (!mi->start) { mesh_index_free(mi); return -1; }
    const double eps = 1e-9;
    for (int pass = 0; pass < 2; ++pass) {
        long long *fill = NULL;
        if (pass == 1) {
            for (long long i = 0; i < nbins; ++i) mi->start[i + 1] += mi->start[i];
            mi->items = (int *)malloc(sizeof(int) * (mi->start[nbins] > 0 ? mi->start[nbins] : 1));
            fill = (long long *)malloc(sizeof(long long) * (nbins + 1));
            if (!mi->items || !fill) { free(fill); mesh_index_free(mi); return -1; }
            memcpy(fill, mi->start, sizeof(long long) * (nbins + 1));
        }
        for (long long e = 0; e < nt; ++e) {
            int blo[3], bhi[3];
            for (int a = 0; a < 3; ++a) {
                double lo = INFINITY, hi = -INFINITY;
                for (int j = 0; j < 4; ++j) {
                    double x = sc->mesh_verts[3 * (long long)sc->mesh_tets[4 * e + j] + a];
                    if (x < lo) lo = x;
                    if (x > hi) hi = x;
                }
                blo[a] = mesh_bin(mi, a, lo - eps);
                bhi[a] = mesh_bin(mi, a, hi + eps);
            }
            for (int z = blo[2]; z <= bhi[2]; ++z)
                for (int y = blo[1]; y <= bhi[1]; ++y)
                    for (int x = blo[0]; x <= bhi[0]; ++x) {
                        long long bin = ((long long)z * mi->r[1] + y) * mi->r[0] + x;
                        if (pass == 0) mi->start[bin + 1]++;
                        else mi->items[fill[bin]++] = (int)e;
                    }
        }
        free(fill);
    }
    return 0;
}

/* Value at p from brick `brick`'s elements; *gap is set when p lies in none of
 * them by more than rounding (smallest barycentric below -1e-5: the elements
 * do not tile the brick). The chosen
 * element and its smallest barycentric coordinate go to *elem and *minb. */
static double sample_mesh(const orc_scene *sc, const mesh_index *mi, int brick, const double p[3],
                          int *gap, long long *elem, double *minb)
{
    const int *items = mi->bitems;
    long long lo = mi->bstart[brick], hi = mi->bstart[brick + 1];
    if (!sc->mesh_bruteforce) {
        long long bin = ((long long)mesh_bin(mi, 2, p[2]) * mi->r[1] + mesh_bin(mi, 1, p[1])) * mi->r[0] +
                        mesh_bin(mi, 0, p[0]);
        items = mi->items;
        lo = mi->start[bin];
        hi = mi->start[bin + 1];
    }
    double best = -INFINITY, val = 0.0;
    long long be = -1;
    for (long long i = lo; i < hi; ++i) {
        const long long e = items[i];
        if (mi->brick[e] != brick) continue;
        double lam[4];
        const double m = tet_bary(sc, e, p, lam);
        if (m > best) {
            best = m;
            be = e;
            val = 0.0;
            for (int j = 0; j < 4; ++j) val += lam[j] * sc->mesh_vals[sc->mesh_tets[4 * e + j]];
        }
    }
    /* float32 vertices on a brick plane lo/Nmax that is not a binary fraction
     * sit up to ~1e-7 of an element off the plane; a real hole is far larger.
     * Outside the domain box (the ambiguity probes take samples up to a few
     * 1e-6 past t_out) the nearest element extends the field, as clamp-to-edge
     * does for voxels. */
    const int inside = p[0] >= 0.0 && p[0] <= mi->E[0] && p[1] >= 0.0 && p[1] <= mi->E[1] && p[2] >= 0.0 &&
                       p[2] <= mi->E[2];
    if (!(best >= -1e-5) && inside) *gap = 1;
    if (elem) *elem = be;
    if (minb) *minb = best;
    return val;
}

/* ---- classification: 1D RGBA transfer function ------------------------
 * Reading (paper silent): u = clamp((s - vmin)/(vmax - vmin), 0, 1) with the
 * global range; entry i of n sits at u = i/(n-1); x = u(n-1),
 * i = min(floor(x), n-2), w = x - i, rgba = (1-w) T[i] + w T[i+1]. The alpha is
 * the opacity of one sample at the configured step (no step correction). */
static double tf_entry(const orc_scene *sc, int i, int c)
{
    return sc->tf64 ? sc->tf64[4 * i + c] : (double)sc->tf[4 * i + c];
}

static void classify(const orc_scene *sc, double s, double rgba[4])
{
    double u = clampd((s - sc->vmin) / (sc->vmax - sc->vmin), 0.0, 1.0);
    double x = u * (sc->ntf - 1);
    int i = (int)floor(x);
    if (i > sc->ntf - 2) i = sc->ntf - 2;
    double w = x - i;
    for (int c = 0; c < 4; ++c)
        rgba[c] = (1.0 - w) * tf_entry(sc, i, c) + w * tf_entry(sc, i + 1, c);
    /* opacity correction (reading; not in the paper): the table holds the
     * opacity of a reference step; a step r times as long keeps the same
     * transmittance per path length: alpha' = 1 - (1 - alpha)^r */
    if (sc->opc_ratio > 0.0 && sc->opc_ratio != 1.0) rgba[3] = 1.0 - pow(1.0 - rgba[3], sc->opc_ratio);
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
    const mesh_index *mi; /* element lists when the scene is a mesh */
    int gap;        /* set when a mesh sample lies in none of its brick's elements */
} pixel_ws;

static double sample_at(const orc_scene *sc, pixel_ws *ws, int brick, const double p[3])
{
    if (sc->mesh_tets) return sample_mesh(sc, ws->mi, brick, p, &ws->gap, NULL, NULL);
    return sample_trilinear(sc, p);
}

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
        double gT = 1.0;
        int gdone = 0;
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
            if (sc->ert_global) {
                /* ray-state cycling (the paper's ray-queue cycling, Sec. 2.2 / 3,
                 * restated for volumes): the ray carries one (C, T) through the
                 * bricks in the order it meets them and stops everywhere once T
                 * falls to the threshold */
                if (gdone) break;
                double rgba[4];
                classify(sc, sample_at(sc, ws, cur, p), rgba);
                for (int ch = 0; ch < 3; ++ch) out[ch] += gT * rgba[3] * rgba[ch];
                gT *= 1.0 - rgba[3];
                ++executed;
                if (ert && gT <= thr) gdone = 1;
                continue;
            }
            if (ws->done[cur]) continue;
            double rgba[4];
            classify(sc, sample_at(sc, ws, cur, p), rgba);
            double Tb = ws->T[cur];
            for (int ch = 0; ch < 3; ++ch) ws->C[3 * cur + ch] += Tb * rgba[3] * rgba[ch];
            ws->T[cur] = Tb * (1.0 - rgba[3]);
            ++executed;
            if (ert && ws->T[cur] <= thr) ws->done[cur] = 1;
        }
        if (sc->ert_global) {
            out[3] = 1.0 - gT;
            goto partials;
        }
        /* front-to-back order along this ray = order of first owned sample */
        {
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
    }
partials:
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
 * a sample fell in a cell that no brick covers (the boxes do not tile), -5 if
 * a mesh sample lay in none of its brick's elements (they do not tile it). */
int orc_render_pixels(const orc_scene *sc, int m, const int *pix, double *img,
                      double *partials, long long *nsamples, int nthreads)
{
    if (!sc || sc->nb < 1 || sc->ntf < 2 || !(sc->vmax > sc->vmin) || sc->step_voxels <= 0)
        return -2;
    long long total = 0;
    int fail = 0;
    if (nthreads < 1) nthreads = 1;
    mesh_index mi;
    memset(&mi, 0, sizeof(mi));
    if (sc->mesh_tets) {
        int rc = mesh_index_build(sc, &mi);
        if (rc) return rc;
    }
#pragma omp parallel num_threads(nthreads) reduction(+ : total) reduction(| : fail)
    {
        pixel_ws ws;
        ws.mi = &mi;
        ws.gap = 0;
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
            if (ws.gap) fail |= 4;
        }
        free(ws.C); free(ws.T); free(ws.first); free(ws.done); free(ws.order);
    }
    mesh_index_free(&mi);
    if (nsamples) *nsamples = total;
    if (fail & 1) return -1;
    if (fail & 2) return -4;
    return (fail & 4) ? -5 : 0;
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

/* ---- gradients (vector-Jacobian product of the rendered pixels) ---------
 * For pixels (m x 2) and an upstream gradient G (m x 4, dL/dI per channel),
 * adds dL/dT (the ntf x 4 table) to grad_tf and dL/dv (every voxel, x fastest)
 * to grad_vol (may be NULL). Early termination must be off. The derivation is
 * the chain rule through the readings above, written out step by step:
 *   composite: I = C_front + F_b (C_b + (1 - A_b) R_b), with F_b the
 *     transmittance in front of brick b and (R_b, 1 - Tb_b) the composite of the
 *     bricks behind it, so dI_rgb/dC_b = F_b, dI_rgb/dA_b = -F_b R_b,
 *     dI_A/dA_b = F_b Tb_b;
 *   per brick: C_{k+1} = C_k + T_k a_k c_k, T_{k+1} = T_k (1 - a_k), A = 1 - T_n,
 *     so with lambda_T(n) = -dL/dA and lambda_C = dL/dC:
 *     dL/dc_k = lambda_C T_k a_k, dL/da_k = T_k (lambda_C . c_k) - T_k lambda_T(k+1),
 *     lambda_T(k) = lambda_T(k+1) (1 - a_k) + a_k (lambda_C . c_k);
 *   table: rgba = (1-w) T[i] + w T[i+1] gives dT[i] += (1-w) g, dT[i+1] += w g,
 *     and ds = (g . (T[i+1] - T[i])) (n-1)/(vmax - vmin) where u is not clamped;
 *   trilinear: dv(corner) += ds * weight(corner), on the clamped global indices.
 * This oracle stores every sample of a ray (it is not the checkpointed GPU
 * adjoint); there is no division by a transmittance anywhere. */
typedef struct {
    double p[3], s, x, rgba[4];
    int brick;
} orc_sample_rec;

static void add_grad_tf(const orc_scene *sc, double *grad_tf, double x, const double g[4])
{
    int i = (int)floor(x);
    if (i > sc->ntf - 2) i = sc->ntf - 2;
    double w = x - i;
    for (int c = 0; c < 4; ++c) {
#pragma omp atomic
        grad_tf[4 * i + c] += (1.0 - w) * g[c];
#pragma omp atomic
        grad_tf[4 * (i + 1) + c] += w * g[c];
    }
}

static void add_grad_vol(const orc_scene *sc, double *grad_vol, const double p[3], double ds)
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
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                long long idx = (dz ? i1[2] : i0[2]) * nxy + (dy ? i1[1] : i0[1]) * nx + (dx ? i1[0] : i0[0]);
#pragma omp atomic
                grad_vol[idx] += ds * w;
            }
}

int orc_render_grad(const orc_scene *sc, int m, const int *pix, const double *grad_img, double *grad_tf,
                    double *grad_vol, int nthreads)
{
    if (!sc || sc->nb < 1 || sc->ntf < 2 || !(sc->vmax > sc->vmin) || sc->step_voxels <= 0 ||
        sc->ert_alpha < 1.0 || (sc->opc_ratio > 0.0 && sc->opc_ratio != 1.0) || sc->mesh_tets)
        return -2;
    const int nm = nmax3(sc->dims);
    const double E[3] = {(double)sc->dims[0] / nm, (double)sc->dims[1] / nm, (double)sc->dims[2] / nm};
    const double dt = sc->step_voxels / nm;
    const double dxds = (sc->ntf - 1) / (sc->vmax - sc->vmin);
    int fail = 0;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads) reduction(| : fail)
    {
        long long cap = 1024;
        orc_sample_rec *rec = (orc_sample_rec *)malloc(sizeof(orc_sample_rec) * cap);
        int *first = (int *)malloc(sizeof(int) * (sc->nb + 1)); /* run start per visited brick */
        int *bid = (int *)malloc(sizeof(int) * (sc->nb + 1));
        double *Cb = (double *)malloc(sizeof(double) * 3 * sc->nb), *Ab = (double *)malloc(sizeof(double) * sc->nb);
        double *Tk = NULL;
        long long tk_cap = 0;
        if (!rec || !first || !bid || !Cb || !Ab) fail = 1;
#pragma omp for schedule(dynamic, 8)
        for (int q = 0; q < m; ++q) {
            if (fail) continue;
            double o[3], d[3], t_in, t_out;
            primary_ray(&sc->cam, pix[2 * q], pix[2 * q + 1], o, d);
            if (!volume_interval(E, o, d, &t_in, &t_out)) continue;
            /* samples in ray order with their owners; owners form contiguous runs */
            long long n = 0;
            int runs = 0, cur = 0;
            for (long long k = 0;; ++k) {
                double t = t_in + (k + 0.5) * dt;
                if (!(t < t_out)) break;
                if (n == cap) {
                    cap *= 2;
                    orc_sample_rec *r2 = (orc_sample_rec *)realloc(rec, sizeof(orc_sample_rec) * cap);
                    if (!r2) { fail = 1; break; }
                    rec = r2;
                }
                orc_sample_rec *r = rec + n;
                int c[3];
                for (int a = 0; a < 3; ++a) {
                    r->p[a] = o[a] + t * d[a];
                    c[a] = clampi((long long)floor(r->p[a] * nm), 0, sc->dims[a] - 1);
                }
                if (!in_box(sc->boxes + 6 * cur, c)) {
                    cur = -1;
                    for (int b = 0; b < sc->nb; ++b)
                        if (in_box(sc->boxes + 6 * b, c)) { cur = b; break; }
                    if (cur < 0) { fail = 2; break; }
                }
                if (runs == 0 || bid[runs - 1] != cur) {
                    if (runs == sc->nb) { fail = 2; break; } /* a brick met twice: boxes not convex */
                    bid[runs] = cur;
                    first[runs] = (int)n;
                    ++runs;
                }
                r->brick = cur;
                r->s = sample_trilinear(sc, r->p);
                r->x = clampd((r->s - sc->vmin) / (sc->vmax - sc->vmin), 0.0, 1.0) * (sc->ntf - 1);
                classify(sc, r->s, r->rgba);
                ++n;
            }
            if (fail) continue;
            first[runs] = (int)n;
            if (n > tk_cap) {
                free(Tk);
                tk_cap = n + 1;
                Tk = (double *)malloc(sizeof(double) * tk_cap);
                if (!Tk) { fail = 1; continue; }
            }
            /* forward per run: T_k and the partial (C, A) */
            for (int j = 0; j < runs; ++j) {
                double C[3] = {0, 0, 0}, T = 1.0;
                for (int k = first[j]; k < first[j + 1]; ++k) {
                    Tk[k] = T;
                    const double *g = rec[k].rgba;
                    for (int ch = 0; ch < 3; ++ch) C[ch] += T * g[3] * g[ch];
                    T *= 1.0 - g[3];
                }
                for (int ch = 0; ch < 3; ++ch) Cb[3 * j + ch] = C[ch];
                Ab[j] = 1.0 - T;
            }
            /* composite adjoint: front transmittance F (forward sweep), behind
             * composite (R, Tb) (backward sweep) */
            const double *G = grad_img + 4 * (long long)q;
            double R[3] = {0, 0, 0}, Tb = 1.0;
            for (int j = runs - 1; j >= 0; --j) {
                double F = 1.0;
                for (int a = 0; a < j; ++a) F *= 1.0 - Ab[a];
                double gC[3] = {F * G[0], F * G[1], F * G[2]};
                double gA = F * (G[3] * Tb - (G[0] * R[0] + G[1] * R[1] + G[2] * R[2]));
                /* per-brick adjoint, back to front */
                double lamT = -gA;
                for (int k = first[j + 1] - 1; k >= first[j]; --k) {
                    const double *c = rec[k].rgba;
                    double a = c[3], Tkk = Tk[k];
                    double gdotc = gC[0] * c[0] + gC[1] * c[1] + gC[2] * c[2];
                    double g[4] = {gC[0] * Tkk * a, gC[1] * Tkk * a, gC[2] * Tkk * a, Tkk * gdotc - Tkk * lamT};
                    lamT = lamT * (1.0 - a) + a * gdotc;
                    if (grad_tf) add_grad_tf(sc, grad_tf, rec[k].x, g);
                    double u = (rec[k].s - sc->vmin) / (sc->vmax - sc->vmin);
                    if (grad_vol && u > 0.0 && u < 1.0) {
                        int i = (int)floor(rec[k].x);
                        if (i > sc->ntf - 2) i = sc->ntf - 2;
                        double ds = 0.0;
                        for (int ch = 0; ch < 4; ++ch) ds += g[ch] * (tf_entry(sc, i + 1, ch) - tf_entry(sc, i, ch));
                        add_grad_vol(sc, grad_vol, rec[k].p, ds * dxds);
                    }
                }
                for (int ch = 0; ch < 3; ++ch) R[ch] = Cb[3 * j + ch] + (1.0 - Ab[j]) * R[ch];
                Tb *= 1.0 - Ab[j];
            }
        }
        free(rec); free(first); free(bid); free(Cb); free(Ab); free(Tk);
    }
    return fail == 0 ? 0 : (fail & 1 ? -1 : -4);
}

/* Mesh point probe: for m world points, the owner brick (cell rule), the value
 * from that brick's elements, the chosen element and its smallest barycentric
 * coordinate. Returns 0, -1/-2 as mesh_index_build, -4 if a point's cell lies in
 * no brick. */
int orc_mesh_sample(const orc_scene *sc, int m, const double *pts, double *vals, long long *elem,
                    double *minb, int *brick)
{
    if (!sc || !sc->mesh_tets) return -2;
    mesh_index mi;
    int rc = mesh_index_build(sc, &mi);
    if (rc) return rc;
    const int nm = nmax3(sc->dims);
    for (int i = 0; i < m; ++i) {
        const double *p = pts + 3 * (long long)i;
        int c[3], b = -1, gap = 0;
        for (int a = 0; a < 3; ++a) c[a] = clampi((long long)floor(p[a] * nm), 0, sc->dims[a] - 1);
        for (int j = 0; j < sc->nb; ++j)
            if (in_box(sc->boxes + 6 * j, c)) { b = j; break; }
        if (b < 0) { rc = -4; break; }
        brick[i] = b;
        vals[i] = sample_mesh(sc, &mi, b, p, &gap, elem + i, minb + i);
    }
    mesh_index_free(&mi);
    return rc;
}

/* Point probes of the two per-sample stages, for function-level pins. */
double orc_sample(const orc_scene *sc, const double p[3]) { return sample_trilinear(sc, p); }
void orc_classify(const orc_scene *sc, double s, double rgba[4]) { classify(sc, s, rgba); }
void orc_primary_ray(const orc_camera *cam, int px, int py, double o[3], double d[3])
{
    primary_ray(cam, px, py, o, d);
}

int orc_version(void) { return 1; }

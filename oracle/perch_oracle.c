/*
 * PERCH 2.0 hypothesis scoring -- plain, slow CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity reference for the CUDA
 * path.  Only the tests, the smoke check and the CPU-baseline leg of the bench
 * may load it; the product library never links, calls or falls back to it, and
 * it shares no code, header or table with the CUDA sources.
 *
 * What it computes, per object-pose hypothesis h (Sec. III-B Eq. 1-2,
 * Sec. IV-A "Parallel Rendering" / "Parallel Cost Computation", Eq. 3,
 * Sec. IV-B Eq. 4, Sec. V-C):
 *   render the mesh at h into an integer depth z-buffer, back-project the
 *   visible pixels, drop those hidden behind the observed depth (R \ C), and
 *   classify each remaining rendered point q against the observed cloud I:
 *   q is explained iff its nearest observed neighbour p lies within delta
 *   (Eq. 2) and, with the colour check on, the CIEDE2000 difference of the two
 *   colours is at most tau_c (Eq. 4).  J_r counts the unexplained q.  Each
 *   observed p inside the admissible set V(h) is an inlier iff it was found as
 *   the nearest neighbour of an explained q (the J_o kernel of Sec. IV-A);
 *   J_o counts the others.
 *
 * Every float line is one IEEE binary32 operation, evaluated in the order
 * written, with no contraction (build with -ffp-contract=off, no fast-math);
 * integer rounding is rintf/llrintf (ties to even).  Edge functions are exact
 * integers (int64 here; their magnitude stays below 2^31 by the guard band).
 * Nearest neighbours are found by brute force over all of I (Eq. 2 as
 * written).  Colour conversion and CIEDE2000 are evaluated in binary32 with
 * the C library's float functions -- the same precision as the CUDA path --
 * and every rendered point whose colour difference lies within 1e-3 of tau_c,
 * or whose hue difference lies within 1e-3 degree of the 180-degree wrap, is
 * counted in a per-hypothesis band report.
 *
 * Readings of the paper (it is silent on these): pixel centres at integer
 * coordinates; 4 sub-pixel bits; no clipping (triangles with a vertex nearer
 * than z_near or outside [-W,2W)x[-H,2H) are culled whole); two-sided
 * rasterisation; top-left style tie rule; perspective-correct depth
 * z = A / sum(w_i / Z_i);
 * nearest depth wins, then lowest triangle id; affine integer colour
 * interpolation; occluder margin m; nearest-neighbour ties to the lowest pixel
 * index; V(h) is the object's inscribed cylinder about its z axis, or
 * labels == object label inside the ROI when labels are used (Sec. V-C).
 *
 * The last section refines hypotheses by M2M GICP (Sec. IV-A) before they
 * are rendered again; its readings are listed there.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_EMPTY UINT64_MAX
#define OR_NWORK 8

typedef struct {
    int32_t W, H;
    float fx, fy, cx, cy;
    const uint16_t *depth;    /* H*W, 0.1 mm units, 0 = invalid            */
    const uint8_t *rgb;       /* H*W*3                                      */
    const int32_t *labels;    /* H*W or NULL                                */
    float delta;              /* metres                                     */
    float tau_c;              /* CIEDE2000 threshold                        */
    int32_t color_check;      /* 0/1                                        */
    int32_t stride;           /* image-space downsampling factor s >= 1     */
    int32_t occ_margin;       /* occluder margin m, 0.1 mm; < 0: no occluder marking (2.0-A) */
    float z_near;             /* metres                                     */
    int32_t jo_mode;          /* 0: NN marks (Sec. IV-A kernel); 1: Eq. 3 as written (Eq. 2 / Eq. 4 from p) */
} or_scene;

typedef struct {
    const float *verts;       /* V*3 object frame, metres                   */
    const uint8_t *rgb;       /* V*3                                        */
    int32_t n_verts;
    const int32_t *tris;      /* T*3                                        */
    int32_t n_tris;
    float vol_r, vol_h;       /* admissible cylinder                        */
} or_mesh;

/* ---------------------------------------------------------------------- */
/* colour: sRGB (IEC 61966-2-1) -> XYZ (D65) -> CIELAB, binary32           */
/* ---------------------------------------------------------------------- */

static float srgb_to_linear(uint8_t c8)
{
    float c = (float)c8 / 255.0f;
    if (c <= 0.04045f)
        return c / 12.92f;
    return powf((c + 0.055f) / 1.055f, 2.4f);
}

static float lab_f(float t)
{
    const float eps = 216.0f / 24389.0f;     /* (6/29)^3            */
    const float kappa = 24389.0f / 27.0f;    /* (29/3)^3            */
    if (t > eps)
        return cbrtf(t);
    return (kappa * t + 16.0f) / 116.0f;
}

void or_srgb_to_lab(const uint8_t rgb[3], float lab[3])
{
    float r = srgb_to_linear(rgb[0]);
    float g = srgb_to_linear(rgb[1]);
    float b = srgb_to_linear(rgb[2]);
    float X = (0.4124564f * r + 0.3575761f * g) + 0.1804375f * b;
    float Y = (0.2126729f * r + 0.7151522f * g) + 0.0721750f * b;
    float Z = (0.0193339f * r + 0.1191920f * g) + 0.9503041f * b;
    float fx = lab_f(X / 0.95047f);
    float fy = lab_f(Y / 1.00000f);
    float fz = lab_f(Z / 1.08883f);
    lab[0] = 116.0f * fy - 16.0f;
    lab[1] = 500.0f * (fx - fy);
    lab[2] = 200.0f * (fy - fz);
}

/* CIEDE2000 colour difference (kL = kC = kH = 1), binary32.  The optional
 * output wrap_gap is | |h1' - h2'| - 180 deg | in degrees (or 1e9 when a
 * chroma is zero), used for the hue-wrap band. */
float or_ciede2000(const float lab1[3], const float lab2[3], float *wrap_gap)
{
    const float PI = 3.14159265358979f;
    const float DEG = PI / 180.0f;
    const float P25_7 = 6103515625.0f;     /* 25^7 */
    float L1 = lab1[0], a1 = lab1[1], b1 = lab1[2];
    float L2 = lab2[0], a2 = lab2[1], b2 = lab2[2];

    float C1 = sqrtf(a1 * a1 + b1 * b1);
    float C2 = sqrtf(a2 * a2 + b2 * b2);
    float Cb = (C1 + C2) / 2.0f;
    float Cb7 = Cb * Cb * Cb * Cb * Cb * Cb * Cb;
    float G = 0.5f * (1.0f - sqrtf(Cb7 / (Cb7 + P25_7)));
    float a1p = (1.0f + G) * a1;
    float a2p = (1.0f + G) * a2;
    float C1p = sqrtf(a1p * a1p + b1 * b1);
    float C2p = sqrtf(a2p * a2p + b2 * b2);

    float h1p = (a1p == 0.0f && b1 == 0.0f) ? 0.0f : atan2f(b1, a1p);
    if (h1p < 0.0f) h1p += 2.0f * PI;
    float h2p = (a2p == 0.0f && b2 == 0.0f) ? 0.0f : atan2f(b2, a2p);
    if (h2p < 0.0f) h2p += 2.0f * PI;

    float dLp = L2 - L1;
    float dCp = C2p - C1p;
    float CC = C1p * C2p;
    float dhp = 0.0f;
    if (CC != 0.0f) {
        dhp = h2p - h1p;
        if (dhp > PI) dhp -= 2.0f * PI;
        else if (dhp < -PI) dhp += 2.0f * PI;
    }
    float dHp = 2.0f * sqrtf(CC) * sinf(dhp / 2.0f);

    float Lbp = (L1 + L2) / 2.0f;
    float Cbp = (C1p + C2p) / 2.0f;
    float hbp;
    if (CC == 0.0f)
        hbp = h1p + h2p;
    else if (fabsf(h1p - h2p) <= PI)
        hbp = (h1p + h2p) / 2.0f;
    else if (h1p + h2p < 2.0f * PI)
        hbp = (h1p + h2p + 2.0f * PI) / 2.0f;
    else
        hbp = (h1p + h2p - 2.0f * PI) / 2.0f;
    if (wrap_gap)
        *wrap_gap = (CC == 0.0f) ? 1e9f : fabsf(fabsf(h1p - h2p) - PI) / DEG;

    float T = 1.0f - 0.17f * cosf(hbp - 30.0f * DEG) + 0.24f * cosf(2.0f * hbp)
              + 0.32f * cosf(3.0f * hbp + 6.0f * DEG) - 0.20f * cosf(4.0f * hbp - 63.0f * DEG);
    float hdeg = hbp / DEG;
    float q = (hdeg - 275.0f) / 25.0f;
    float dtheta = 30.0f * DEG * expf(-(q * q));
    float Cbp7 = Cbp * Cbp * Cbp * Cbp * Cbp * Cbp * Cbp;
    float RC = 2.0f * sqrtf(Cbp7 / (Cbp7 + P25_7));
    float l50 = (Lbp - 50.0f) * (Lbp - 50.0f);
    float SL = 1.0f + 0.015f * l50 / sqrtf(20.0f + l50);
    float SC = 1.0f + 0.045f * Cbp;
    float SH = 1.0f + 0.015f * Cbp * T;
    float RT = -sinf(2.0f * dtheta) * RC;
    float tL = dLp / SL, tC = dCp / SC, tH = dHp / SH;
    return sqrtf(tL * tL + tC * tC + tH * tH + RT * tC * tH);
}

/* ---------------------------------------------------------------------- */
/* rasterisation                                                           */
/* ---------------------------------------------------------------------- */

/* Edge function E(a,b,p) = (b.x-a.x)(p.y-a.y) - (b.y-a.y)(p.x-a.x). */
static int64_t edge(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t px, int64_t py)
{
    return (bx - ax) * (py - ay) - (by - ay) * (px - ax);
}

/* An edge with direction (dx,dy) owns the samples lying exactly on it iff
 * dy > 0, or dy == 0 and dx < 0. */
static int owns_edge(int64_t dx, int64_t dy)
{
    return dy > 0 || (dy == 0 && dx < 0);
}

static int64_t floor_div16(int64_t x) { return x >= 0 ? x / 16 : -((-x + 15) / 16); }
static int64_t ceil_div16(int64_t x) { return -floor_div16(-x); }

/* Screen-space set-up of one triangle at a pose: returns 0 if culled or
 * degenerate.  xs/ys are the snapped vertex positions (1/16 px), iz = 1/Z,
 * vid the mesh vertex ids after the orientation swap, A > 0 the doubled area. */
typedef struct {
    int64_t xs[3], ys[3];
    float iz[3];
    int32_t vid[3];
    int64_t A;
} or_tri;

static int setup_triangle(const or_scene *sc, const or_mesh *m, const float *P, int32_t t,
                          or_tri *o, int *culled)
{
    *culled = 0;
    for (int k = 0; k < 3; k++) {
        int32_t vi = m->tris[3 * t + k];
        float vx = m->verts[3 * vi + 0], vy = m->verts[3 * vi + 1], vz = m->verts[3 * vi + 2];
        /* C1: X = R v + t */
        float X = ((P[0] * vx + P[1] * vy) + P[2] * vz) + P[3];
        float Y = ((P[4] * vx + P[5] * vy) + P[6] * vz) + P[7];
        float Z = ((P[8] * vx + P[9] * vy) + P[10] * vz) + P[11];
        if (!(Z >= sc->z_near)) { *culled = 1; return 0; }
        /* C2: pinhole projection, 4 sub-pixel bits */
        float px = sc->fx * (X / Z) + sc->cx;
        float py = sc->fy * (Y / Z) + sc->cy;
        float sx = px * 16.0f;
        float sy = py * 16.0f;
        if (!(sx >= (float)(-16 * sc->W)) || !(sx < (float)(32 * sc->W)) ||
            !(sy >= (float)(-16 * sc->H)) || !(sy < (float)(32 * sc->H))) {
            *culled = 1;
            return 0;
        }
        o->xs[k] = (int64_t)llrintf(sx);
        o->ys[k] = (int64_t)llrintf(sy);
        o->iz[k] = 1.0f / Z;
        o->vid[k] = vi;
    }
    int64_t A = edge(o->xs[0], o->ys[0], o->xs[1], o->ys[1], o->xs[2], o->ys[2]);
    if (A == 0)
        return 0;
    if (A < 0) {   /* two-sided: swap b and c */
        int64_t tx = o->xs[1], ty = o->ys[1];
        float ti = o->iz[1];
        int32_t tv = o->vid[1];
        o->xs[1] = o->xs[2]; o->ys[1] = o->ys[2]; o->iz[1] = o->iz[2]; o->vid[1] = o->vid[2];
        o->xs[2] = tx; o->ys[2] = ty; o->iz[2] = ti; o->vid[2] = tv;
        A = -A;
    }
    o->A = A;
    return 1;
}

/* Edge values (w0,w1,w2) of pixel (u,v); returns 1 iff the sample is covered. */
static int coverage(const or_tri *o, int64_t u, int64_t v, int64_t w[3])
{
    int64_t sx = 16 * u, sy = 16 * v;
    const int64_t *x = o->xs, *y = o->ys;
    w[0] = edge(x[1], y[1], x[2], y[2], sx, sy);   /* edge b -> c */
    w[1] = edge(x[2], y[2], x[0], y[0], sx, sy);   /* edge c -> a */
    w[2] = edge(x[0], y[0], x[1], y[1], sx, sy);   /* edge a -> b */
    int64_t dxs[3] = {x[2] - x[1], x[0] - x[2], x[1] - x[0]};
    int64_t dys[3] = {y[2] - y[1], y[0] - y[2], y[1] - y[0]};
    for (int i = 0; i < 3; i++) {
        if (w[i] > 0)
            continue;
        if (w[i] == 0 && owns_edge(dxs[i], dys[i]))
            continue;
        return 0;
    }
    return 1;
}

static void clip_roi(const or_scene *sc, const int32_t roi[4], int64_t *u0, int64_t *v0,
                     int64_t *u1, int64_t *v1)
{
    *u0 = roi[0] > 0 ? roi[0] : 0;
    *v0 = roi[1] > 0 ? roi[1] : 0;
    *u1 = roi[2] < sc->W ? roi[2] : sc->W;
    *v1 = roi[3] < sc->H ? roi[3] : sc->H;
}

/* Render one hypothesis into keys[H*W]: key = (d << 32) | triangle id, the
 * smallest key wins (nearest depth, then lowest id); OR_EMPTY where nothing
 * covers.  work (may be NULL) accumulates [setups, culled, fragments]. */
int or_render_keys(const or_scene *sc, const or_mesh *m, const float pose[12],
                   const int32_t roi[4], uint64_t *keys, int64_t *work)
{
    int64_t W = sc->W, H = sc->H;
    for (int64_t i = 0; i < W * H; i++)
        keys[i] = OR_EMPTY;
    int64_t ru0, rv0, ru1, rv1;
    clip_roi(sc, roi, &ru0, &rv0, &ru1, &rv1);
    for (int32_t t = 0; t < m->n_tris; t++) {
        or_tri o;
        int culled;
        if (work) work[0]++;
        if (!setup_triangle(sc, m, pose, t, &o, &culled)) {
            if (work && culled) work[1]++;
            continue;
        }
        int64_t xmin = o.xs[0], xmax = o.xs[0], ymin = o.ys[0], ymax = o.ys[0];
        for (int k = 1; k < 3; k++) {
            if (o.xs[k] < xmin) xmin = o.xs[k];
            if (o.xs[k] > xmax) xmax = o.xs[k];
            if (o.ys[k] < ymin) ymin = o.ys[k];
            if (o.ys[k] > ymax) ymax = o.ys[k];
        }
        int64_t u0 = ceil_div16(xmin), u1 = floor_div16(xmax);
        int64_t v0 = ceil_div16(ymin), v1 = floor_div16(ymax);
        if (u0 < ru0) u0 = ru0;
        if (v0 < rv0) v0 = rv0;
        if (u1 > ru1 - 1) u1 = ru1 - 1;
        if (v1 > rv1 - 1) v1 = rv1 - 1;
        for (int64_t v = v0; v <= v1; v++) {
            for (int64_t u = u0; u <= u1; u++) {
                int64_t w[3];
                if (!coverage(&o, u, v, w))
                    continue;
                /* C4: perspective-correct depth from interpolated 1/Z:
                 * z = A / (w0/Z0 + w1/Z1 + w2/Z2), one division */
                float num = ((float)w[0] * o.iz[0] + (float)w[1] * o.iz[1]) + (float)w[2] * o.iz[2];
                float z = (float)o.A / num;
                float dz = z * 10000.0f;
                if (!(dz < 4294967296.0f))
                    continue;
                int64_t d = (int64_t)llrintf(dz);
                if (d < 1 || d > 4294967295LL)
                    continue;
                if (work) work[2]++;
                uint64_t key = ((uint64_t)d << 32) | (uint64_t)(uint32_t)t;
                if (key < keys[v * W + u])
                    keys[v * W + u] = key;
            }
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* point clouds                                                            */
/* ---------------------------------------------------------------------- */

/* C7: back-projection of pixel (u,v) at integer depth d (0.1 mm). */
static void back_project(const or_scene *sc, int64_t u, int64_t v, int64_t d, float p[3])
{
    float z = (float)d / 10000.0f;
    p[0] = (((float)u - sc->cx) * z) / sc->fx;
    p[1] = (((float)v - sc->cy) * z) / sc->fy;
    p[2] = z;
}

/* The observed cloud I: every valid pixel whose coordinates are multiples of
 * the stride, in increasing pixel index.  xyz (n*3), lab (n*3), pix (n) may be
 * NULL; returns n. */
int64_t or_observed_points(const or_scene *sc, float *xyz, float *lab, int32_t *pix)
{
    int64_t n = 0, s = sc->stride;
    for (int64_t v = 0; v < sc->H; v++)
        for (int64_t u = 0; u < sc->W; u++) {
            int64_t i = v * sc->W + u;
            if (u % s != 0 || v % s != 0 || sc->depth[i] == 0)
                continue;
            if (xyz) back_project(sc, u, v, sc->depth[i], xyz + 3 * n);
            if (lab) or_srgb_to_lab(sc->rgb + 3 * i, lab + 3 * n);
            if (pix) pix[n] = (int32_t)i;
            n++;
        }
    return n;
}

/* Resolve the key buffer of one hypothesis into its rendered cloud R \ C:
 * visible pixels at stride positions that are not hidden behind the observed
 * depth (C5-C7).  Outputs (capacity H*W): xyz n*3, rgb n*3, pix n.  Returns n. */
int64_t or_rendered_points(const or_scene *sc, const or_mesh *m, const float pose[12],
                           int32_t label, const uint64_t *keys, float *xyz, uint8_t *rgb,
                           int32_t *pix)
{
    int64_t n = 0, s = sc->stride;
    for (int64_t v = 0; v < sc->H; v++)
        for (int64_t u = 0; u < sc->W; u++) {
            int64_t i = v * sc->W + u;
            uint64_t key = keys[i];
            if (key == OR_EMPTY || u % s != 0 || v % s != 0)
                continue;
            int64_t d = (int64_t)(key >> 32);
            int32_t t = (int32_t)(key & 0xffffffffu);
            /* C6: occluders -- the observed surface is nearer by more than m */
            int64_t dobs = sc->depth[i];
            if (sc->occ_margin >= 0 && dobs > 0 && dobs + sc->occ_margin < d &&
                (label < 0 || sc->labels == NULL || sc->labels[i] != label))
                continue;
            or_tri o;
            int culled;
            setup_triangle(sc, m, pose, t, &o, &culled);
            int64_t w[3];
            coverage(&o, u, v, w);
            /* C5: affine integer colour, rounded half up */
            for (int k = 0; k < 3; k++) {
                int64_t c = w[0] * m->rgb[3 * o.vid[0] + k] + w[1] * m->rgb[3 * o.vid[1] + k]
                            + w[2] * m->rgb[3 * o.vid[2] + k] + o.A / 2;
                if (rgb) rgb[3 * n + k] = (uint8_t)(c / o.A);
            }
            if (xyz) back_project(sc, u, v, d, xyz + 3 * n);
            if (pix) pix[n] = (int32_t)i;
            n++;
        }
    return n;
}

/* C11: is observed point p (pixel i) in the admissible set V(h)? */
static int in_volume(const or_scene *sc, const or_mesh *m, const float *P, int32_t label,
                     const int32_t roi[4], int64_t i, const float p[3])
{
    if (label >= 0) {
        int64_t u = i % sc->W, v = i / sc->W;
        return sc->labels[i] == label && u >= roi[0] && u < roi[2] && v >= roi[1] && v < roi[3];
    }
    float e0 = p[0] - P[3], e1 = p[1] - P[7], e2 = p[2] - P[11];
    float q0 = (P[0] * e0 + P[4] * e1) + P[8] * e2;    /* R^T (p - t) */
    float q1 = (P[1] * e0 + P[5] * e1) + P[9] * e2;
    float q2 = (P[2] * e0 + P[6] * e1) + P[10] * e2;
    return (q0 * q0 + q1 * q1) <= m->vol_r * m->vol_r && q2 >= 0.0f && q2 <= m->vol_h;
}

/* ---------------------------------------------------------------------- */
/* nearest neighbours: brute force (Eq. 2 as written) or a uniform grid     */
/* ---------------------------------------------------------------------- */
/*
 * The grid mode finds the same nearest neighbour as the brute-force scan in
 * far less time, so that whole configurations can be checked:
 *   cells of edge h = delta (1 + 1/32), cell coordinate floorf(x / h) per
 *   axis; the points (copied) sorted by (cell z, cell y, cell x, index); a
 *   query scans the 3 x 3 x 3 cells around its own.
 * Why that is exact: a point p with fl(d2) <= fl(delta^2) lies within
 * delta (1 + 2^-20) of q on every axis; fl(x / h) is within 2^-8 of x / h
 * for the coordinates accepted here (|x / h| < 2^16), so the cell
 * coordinates of q and p differ by at most
 * floor((1 + 2^-20) / ((1 + 1/32)(1 - 2^-24)) + 2^-7) = floor(0.978) + 1,
 * i.e. by at most one.  Hence the nearest point within delta, if there is
 * one, is among the candidates and is their minimum (same d2 expression, same
 * tie rule: the lowest index); if there is none, no candidate passes the
 * delta test either.  Clouds with a larger coordinate fall back to the brute
 * force.  (The work counter of delta-cell candidates is the brute force's
 * alone.)
 */
#define OR_GRID_BIAS (1 << 20)
#define OR_GRID_LIMIT 65528.0f       /* |x / h| bound, 2^16 - 8 */

typedef struct {
    int64_t key, idx;
    float p[3];                /* the point, copied: the scan reads it in cell order */
} or_cell_entry;

typedef struct {
    or_cell_entry *e;          /* n entries sorted by (key, idx)            */
    int64_t n;
    int usable;                /* 0: some |x / h| too large, brute force    */
    float h;                   /* cell edge                                 */
} or_grid;

static int64_t or_cell_key(int64_t cx, int64_t cy, int64_t cz)
{
    return ((cz + OR_GRID_BIAS) << 42) | ((cy + OR_GRID_BIAS) << 21) | (cx + OR_GRID_BIAS);
}

static int or_cmp_entry(const void *a, const void *b)
{
    const or_cell_entry *x = a, *y = b;
    if (x->key != y->key)
        return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static int or_cell_of(float x, float h, int32_t *c)
{
    float t = x / h;
    if (!(fabsf(t) < OR_GRID_LIMIT))
        return 0;
    *c = (int32_t)floorf(t);
    return 1;
}

/* Build the grid of n points (xyz) into g->e (capacity n). */
static void or_grid_build(or_grid *g, const float *xyz, int64_t n, float delta)
{
    g->n = n;
    g->h = delta * 1.03125f;
    g->usable = g->h > 0.0f;
    for (int64_t j = 0; j < n && g->usable; j++) {
        int32_t c[3];
        for (int a = 0; a < 3 && g->usable; a++)
            g->usable = or_cell_of(xyz[3 * j + a], g->h, &c[a]);
        if (g->usable) {
            g->e[j].key = or_cell_key(c[0], c[1], c[2]);
            g->e[j].idx = j;
            g->e[j].p[0] = xyz[3 * j];
            g->e[j].p[1] = xyz[3 * j + 1];
            g->e[j].p[2] = xyz[3 * j + 2];
        }
    }
    if (g->usable)
        qsort(g->e, (size_t)n, sizeof(or_cell_entry), or_cmp_entry);
}

/* The 9 row ranges [lo, hi) of the sorted entries around the last query
 * cell, reused while consecutive queries fall in the same cell (the
 * rendered points come in pixel order, so most do). */
typedef struct {
    int valid;
    int32_t qc[3];
    int64_t lo[9], hi[9];
} or_grid_cache;

/* First entry with key >= k. */
static int64_t or_lower_bound(const or_grid *g, int64_t k)
{
    int64_t lo = 0, hi = g->n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->e[mid].key < k)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

/* Nearest point of the cloud xyz (n points) to q: smallest
 * d2 = (dx dx + dy dy) + dz dz, ties to the lowest index; returns its index
 * (-1 for an empty cloud) and its d2 in *best_d2.  With a usable grid only
 * the 3 x 3 x 3 cells around q are scanned (exact for every point within
 * delta, see above); otherwise every point, and then cand27 (may be NULL)
 * counts the points whose cells (cells: floorf(x / delta) per point) are
 * within one of q's on every axis. */
static int64_t or_nearest(const float *xyz, int64_t n, const or_grid *g, or_grid_cache *gc,
                          const int32_t *cells, const float q[3], float delta, float *best_d2, int64_t *cand27)
{
    float best = INFINITY;
    int64_t bj = -1;
    int32_t qc[3];
    int use_grid = g && g->usable && or_cell_of(q[0], g->h, &qc[0]) && or_cell_of(q[1], g->h, &qc[1]) &&
                   or_cell_of(q[2], g->h, &qc[2]);
    if (!use_grid) {
        int32_t c0 = (int32_t)floorf(q[0] / delta), c1 = (int32_t)floorf(q[1] / delta),
                c2 = (int32_t)floorf(q[2] / delta);
        for (int64_t j = 0; j < n; j++) {
            const float *p = xyz + 3 * j;
            float dx = q[0] - p[0], dy = q[1] - p[1], dz = q[2] - p[2];
            float d2 = (dx * dx + dy * dy) + dz * dz;
            if (d2 < best) { best = d2; bj = j; }
            if (cand27 && cells) {
                const int32_t *pc = cells + 3 * j;
                if (abs(pc[0] - c0) <= 1 && abs(pc[1] - c1) <= 1 && abs(pc[2] - c2) <= 1)
                    (*cand27)++;
            }
        }
        *best_d2 = best;
        return bj;
    }
    if (!gc->valid || gc->qc[0] != qc[0] || gc->qc[1] != qc[1] || gc->qc[2] != qc[2]) {
        for (int r = 0; r < 9; r++) {
            int dz = r / 3 - 1, dy = r % 3 - 1;
            gc->lo[r] = or_lower_bound(g, or_cell_key(qc[0] - 1, qc[1] + dy, qc[2] + dz));
            gc->hi[r] = or_lower_bound(g, or_cell_key(qc[0] + 1, qc[1] + dy, qc[2] + dz) + 1);
        }
        gc->valid = 1;
        gc->qc[0] = qc[0]; gc->qc[1] = qc[1]; gc->qc[2] = qc[2];
    }
    for (int r = 0; r < 9; r++)
        for (int64_t i = gc->lo[r]; i < gc->hi[r]; i++) {
            int64_t j = g->e[i].idx;
            const float *p = g->e[i].p;
            float dx = q[0] - p[0], dy = q[1] - p[1], dz = q[2] - p[2];
            float d2 = (dx * dx + dy * dy) + dz * dz;
            if (d2 < best || (d2 == best && j < bj)) { best = d2; bj = j; }
        }
    *best_d2 = best;
    return bj;
}

/* ---------------------------------------------------------------------- */
/* scoring                                                                 */
/* ---------------------------------------------------------------------- */

/* Score n hypotheses.  costs[2h] = J_o, costs[2h+1] = J_r.  band[h] (may be
 * NULL) = points whose colour decision lies in the tolerance band: rendered
 * points, and under jo_mode 1 also the observed points of V whose decision
 * against their nearest rendered point does.
 * work[8h..8h+7] (may be NULL) = triangle set-ups, culled triangles,
 * fragments, visible pixels, kept rendered points L, delta-cell candidates
 * (observed points in the 27 cells of edge delta around q's cell), |I cap V|,
 * explained points.  n_threads <= 0 uses the OpenMP default. */
int or_score_nn(const or_scene *sc, const or_mesh *m, int32_t label, const int32_t roi[4],
                const float *poses, int64_t n, int32_t *costs, int32_t *band, int64_t *work,
                int32_t n_threads, int32_t grid)
{
    int64_t WH = (int64_t)sc->W * sc->H;
    float *Ixyz = malloc(sizeof(float) * 3 * (WH + 1));
    float *Ilab = malloc(sizeof(float) * 3 * (WH + 1));
    int32_t *Ipix = malloc(sizeof(int32_t) * (WH + 1));
    or_grid Ig = {NULL, 0, 0, 0.0f};
    if (grid)
        Ig.e = malloc(sizeof(or_cell_entry) * (WH + 1));
    if (!Ixyz || !Ilab || !Ipix || (grid && !Ig.e)) {
        free(Ixyz); free(Ilab); free(Ipix); free(Ig.e);
        return -2;
    }
    int64_t nI = or_observed_points(sc, Ixyz, Ilab, Ipix);
    int32_t *Icell = malloc(sizeof(int32_t) * 3 * (nI + 1));
    if (!Icell) {
        free(Ixyz); free(Ilab); free(Ipix); free(Ig.e);
        return -2;
    }
    for (int64_t j = 0; j < 3 * nI; j++)
        Icell[j] = (int32_t)floorf(Ixyz[j] / sc->delta);
    if (grid)
        or_grid_build(&Ig, Ixyz, nI, sc->delta);
    float delta2 = sc->delta * sc->delta;
    int rc = 0;
#ifdef _OPENMP
    if (n_threads > 0)
        omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel
    {
        uint64_t *keys = malloc(sizeof(uint64_t) * WH);
        float *Rxyz = malloc(sizeof(float) * 3 * WH);
        uint8_t *Rrgb = malloc(3 * WH);
        int32_t *Rpix = malloc(sizeof(int32_t) * WH);
        uint8_t *mark = malloc(nI + 1);
        or_grid Rg = {NULL, 0, 0, 0.0f};
        if (grid && sc->jo_mode == 1)
            Rg.e = malloc(sizeof(or_cell_entry) * (WH + 1));
        int ok = keys && Rxyz && Rrgb && Rpix && mark && (!(grid && sc->jo_mode == 1) || Rg.e);
        if (!ok) {
#pragma omp atomic write
            rc = -2;
        }
        /* every thread reaches the work-sharing loop, even one whose buffers failed */
#pragma omp for schedule(dynamic, 1)
        for (int64_t h = 0; h < n; h++) {
            if (!ok)
                continue;
            {
                const float *P = poses + 12 * h;
                int64_t wk[OR_NWORK] = {0};
                or_render_keys(sc, m, P, roi, keys, wk);
                for (int64_t i = 0; i < WH; i++)
                    wk[3] += keys[i] != OR_EMPTY;
                int64_t L = or_rendered_points(sc, m, P, label, keys, Rxyz, Rrgb, Rpix);
                wk[4] = L;
                memset(mark, 0, nI + 1);
                int32_t Jr = 0, nband = 0;
                or_grid_cache gcache = {0}, rcache = {0};
                for (int64_t k = 0; k < L; k++) {
                    const float *q = Rxyz + 3 * k;
                    float best;
                    /* Eq. 2: nearest neighbour over all of I, ties to lowest index */
                    int64_t bj = or_nearest(Ixyz, nI, grid ? &Ig : NULL, &gcache, Icell, q, sc->delta, &best, &wk[5]);
                    int explained = bj >= 0 && best <= delta2;
                    if (explained && sc->color_check) {
                        /* Eq. 4: colour of q against its nearest neighbour p'' */
                        float lq[3], gap;
                        or_srgb_to_lab(Rrgb + 3 * k, lq);
                        float dE = or_ciede2000(lq, Ilab + 3 * bj, &gap);
                        if (fabsf(dE - sc->tau_c) <= 1e-3f || gap <= 1e-3f)
                            nband++;
                        if (dE > sc->tau_c)
                            explained = 0;
                    }
                    if (explained) {
                        mark[bj] = 1;
                        wk[7]++;
                    } else {
                        Jr++;
                    }
                }
                int32_t Jo = 0;
                if (grid && sc->jo_mode == 1)
                    or_grid_build(&Rg, Rxyz, L, sc->delta);
                for (int64_t j = 0; j < nI; j++) {
                    if (!in_volume(sc, m, P, label, roi, Ipix[j], Ixyz + 3 * j))
                        continue;
                    wk[6]++;
                    if (sc->jo_mode == 1) {
                        /* Eq. 3 as written: OUTLIER(p | R \ C), with Eq. 2 / Eq. 4
                         * applied from the observed side ("or vice-versa",
                         * Sec. IV-B): p's nearest rendered point q'' (smallest
                         * d2, ties to the lowest pixel index -- R is listed in
                         * pixel order) must lie within delta and, with the colour
                         * check on, differ from p by at most tau_c. */
                        const float *p = Ixyz + 3 * j;
                        float best;
                        int64_t bk = or_nearest(Rxyz, L, grid ? &Rg : NULL, &rcache, NULL, p, sc->delta, &best, NULL);
                        int inlier = bk >= 0 && best <= delta2;
                        if (inlier && sc->color_check) {
                            float lq[3], gap;
                            or_srgb_to_lab(Rrgb + 3 * bk, lq);
                            float dE = or_ciede2000(lq, Ilab + 3 * j, &gap);
                            if (fabsf(dE - sc->tau_c) <= 1e-3f || gap <= 1e-3f)
                                nband++;
                            if (dE > sc->tau_c)
                                inlier = 0;
                        }
                        if (!inlier)
                            Jo++;
                    } else if (!mark[j]) {
                        Jo++;
                    }
                }
                costs[2 * h] = Jo;
                costs[2 * h + 1] = Jr;
                if (band) band[h] = nband;
                if (work)
                    memcpy(work + OR_NWORK * h, wk, sizeof(wk));
            }
        }
        free(keys); free(Rxyz); free(Rrgb); free(Rpix); free(mark); free(Rg.e);
    }
    free(Ixyz); free(Ilab); free(Ipix); free(Icell); free(Ig.e);
    return rc;
}

/* or_score_nn with the brute-force nearest neighbours (Eq. 2 as written). */
int or_score(const or_scene *sc, const or_mesh *m, int32_t label, const int32_t roi[4],
             const float *poses, int64_t n, int32_t *costs, int32_t *band, int64_t *work,
             int32_t n_threads)
{
    return or_score_nn(sc, m, label, roi, poses, n, costs, band, work, n_threads, 0);
}

/* C12: J = J_o + J_r; best = minimum J, ties to the lowest id (ids NULL: the
 * index).  Returns -1 if n < 1. */
int or_best(const int32_t *costs, const uint64_t *ids, int64_t n, int64_t *best_index,
            int32_t *best_cost)
{
    if (n < 1)
        return -1;
    int64_t bi = 0;
    int64_t bJ = (int64_t)costs[0] + costs[1];
    for (int64_t h = 1; h < n; h++) {
        int64_t J = (int64_t)costs[2 * h] + costs[2 * h + 1];
        uint64_t idh = ids ? ids[h] : (uint64_t)h;
        uint64_t idb = ids ? ids[bi] : (uint64_t)bi;
        if (J < bJ || (J == bJ && idh < idb)) {
            bJ = J;
            bi = h;
        }
    }
    *best_index = bi;
    *best_cost = (int32_t)bJ;
    return 0;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* M2M GICP refinement (Sec. IV-A "Parallel M2M GICP"; Sec. III-A: local   */
/* ICP adjusts each successor's pose before it is rendered again)          */
/* ---------------------------------------------------------------------- */
/*
 * Source: the rendered cloud R \ C of the hypothesis at its input pose (the
 * kept points of the scorer), each point carrying the unit normal of the
 * triangle it was rendered from.  Target: the observed cloud I with a normal
 * per pixel from central differences of the depth image.  GICP models every
 * point as a Gaussian flattened along its surface normal,
 * C(n) = I - (1 - eps) n n^T (a zero normal gives C = I), and minimises
 * sum_i r_i^T (C_b + R C_a R^T)^-1 r_i over a rigid increment by
 * Gauss-Newton, with r = b - (R a + t) for the nearest observed point b
 * within delta of the moved source point.
 *
 * Readings (the paper names the method and its GPU parts only): covariances
 * from the exact surface (mesh triangle) and from image-space neighbours;
 * a fixed correspondence radius delta (the hash radius of the observation);
 * the increment linearised as (I + [w]x) p + v; per-correspondence terms in
 * binary32 in the order written, quantised to integer multiples of 2^-24
 * and summed exactly in int64 (so that any summation order gives the same
 * sums); the 6x6 system solved by Cholesky in binary64; the rotation update
 * from the quaternion (1, w/2) normalised (rational operations and one square
 * root).  Iteration stops after max_iters updates, when a step is below the
 * thresholds, with fewer than min_corr correspondences, or when the system
 * is not positive definite.
 */

#define OR_GICP_NVAL 28        /* H upper triangle (21), g (6), sum r^T M r (1) */
#define OR_GICP_SCALE 16777216.0f
#define OR_GICP_LIMIT 1048576.0f   /* |term| bound: a point beyond it is skipped */

typedef struct {
    int32_t max_iters;
    float epsilon;            /* plane regulariser of the covariances     */
    int32_t normal_jump;      /* max |d_neighbour - d_centre|, 0.1 mm     */
    int32_t min_corr;
    float stop_rot;           /* radians                                  */
    float stop_trans;         /* metres                                   */
} or_gicp_params;

/* Unit normal of mesh triangle t in the object frame (vertex order as
 * stored): normalise((v1 - v0) x (v2 - v0)); zero for a degenerate one. */
void or_triangle_normal(const or_mesh *m, int32_t t, float n[3])
{
    const float *a = m->verts + 3 * m->tris[3 * t + 0];
    const float *b = m->verts + 3 * m->tris[3 * t + 1];
    const float *c = m->verts + 3 * m->tris[3 * t + 2];
    float e1x = b[0] - a[0], e1y = b[1] - a[1], e1z = b[2] - a[2];
    float e2x = c[0] - a[0], e2y = c[1] - a[1], e2z = c[2] - a[2];
    float cx = e1y * e2z - e1z * e2y;
    float cy = e1z * e2x - e1x * e2z;
    float cz = e1x * e2y - e1y * e2x;
    float len2 = (cx * cx + cy * cy) + cz * cz;
    if (!(len2 > 0.0f)) {
        n[0] = n[1] = n[2] = 0.0f;
        return;
    }
    float inv = 1.0f / sqrtf(len2);
    n[0] = cx * inv;
    n[1] = cy * inv;
    n[2] = cz * inv;
}

/* Normal of the observed surface at pixel (u, v): the cross product of the
 * central differences P(u+1,v) - P(u-1,v) and P(u,v+1) - P(u,v-1) of the
 * back-projected depth, normalised.  Zero when the pixel or one of its four
 * neighbours is outside the image, has no depth, or differs from the centre
 * depth by more than normal_jump. */
void or_observed_normal(const or_scene *sc, int32_t normal_jump, int64_t u, int64_t v, float n[3])
{
    n[0] = n[1] = n[2] = 0.0f;
    if (u < 1 || v < 1 || u + 1 >= sc->W || v + 1 >= sc->H)
        return;
    int64_t W = sc->W;
    int64_t dc = sc->depth[v * W + u];
    int64_t du[4] = {u - 1, u + 1, u, u};
    int64_t dv[4] = {v, v, v - 1, v + 1};
    float P[4][3];
    if (dc == 0)
        return;
    for (int k = 0; k < 4; k++) {
        int64_t d = sc->depth[dv[k] * W + du[k]];
        if (d == 0 || llabs(d - dc) > normal_jump)
            return;
        back_project(sc, du[k], dv[k], d, P[k]);
    }
    float ax = P[1][0] - P[0][0], ay = P[1][1] - P[0][1], az = P[1][2] - P[0][2];
    float bx = P[3][0] - P[2][0], by = P[3][1] - P[2][1], bz = P[3][2] - P[2][2];
    float cx = ay * bz - az * by;
    float cy = az * bx - ax * bz;
    float cz = ax * by - ay * bx;
    float len2 = (cx * cx + cy * cy) + cz * cz;
    if (!(len2 > 0.0f))
        return;
    float inv = 1.0f / sqrtf(len2);
    n[0] = cx * inv;
    n[1] = cy * inv;
    n[2] = cz * inv;
}

/* The 28 binary32 terms of one correspondence: source point a with normal na
 * moved by (Rf, tf) to p, matched to observed b with normal nb.  Returns 0
 * (no terms) when the combined covariance is not positive or a term exceeds
 * the bound.  Term order: H(0,0..5), H(1,1..5), ..., H(5,5), g(0..5), r^T M r. */
int or_gicp_terms(const float Rf[9], const float tf[3], const float a[3], const float na[3],
                  const float b[3], const float nb[3], float eps, float out[OR_GICP_NVAL])
{
    float p0 = ((Rf[0] * a[0] + Rf[1] * a[1]) + Rf[2] * a[2]) + tf[0];
    float p1 = ((Rf[3] * a[0] + Rf[4] * a[1]) + Rf[5] * a[2]) + tf[1];
    float p2 = ((Rf[6] * a[0] + Rf[7] * a[1]) + Rf[8] * a[2]) + tf[2];
    float m0 = (Rf[0] * na[0] + Rf[1] * na[1]) + Rf[2] * na[2];
    float m1 = (Rf[3] * na[0] + Rf[4] * na[1]) + Rf[5] * na[2];
    float m2 = (Rf[6] * na[0] + Rf[7] * na[1]) + Rf[8] * na[2];
    float e = 1.0f - eps;
    /* C = 2 I - e (nb nb^T + m m^T) */
    float c00 = 2.0f - e * (nb[0] * nb[0] + m0 * m0);
    float c11 = 2.0f - e * (nb[1] * nb[1] + m1 * m1);
    float c22 = 2.0f - e * (nb[2] * nb[2] + m2 * m2);
    float c01 = -(e * (nb[0] * nb[1] + m0 * m1));
    float c02 = -(e * (nb[0] * nb[2] + m0 * m2));
    float c12 = -(e * (nb[1] * nb[2] + m1 * m2));
    /* M = C^-1 by the adjugate */
    float a00 = c11 * c22 - c12 * c12;
    float a01 = c02 * c12 - c01 * c22;
    float a02 = c01 * c12 - c02 * c11;
    float a11 = c00 * c22 - c02 * c02;
    float a12 = c01 * c02 - c00 * c12;
    float a22 = c00 * c11 - c01 * c01;
    float det = (c00 * a00 + c01 * a01) + c02 * a02;
    if (!(det > 0.0f))
        return 0;
    float id = 1.0f / det;
    float M[3][3];
    M[0][0] = a00 * id; M[0][1] = a01 * id; M[0][2] = a02 * id;
    M[1][0] = M[0][1];  M[1][1] = a11 * id; M[1][2] = a12 * id;
    M[2][0] = M[0][2];  M[2][1] = M[1][2];  M[2][2] = a22 * id;
    float r[3] = {b[0] - p0, b[1] - p1, b[2] - p2};
    /* Jacobian of r w.r.t. (w, v): [ [p]x , -I ]; MA = M [p]x */
    float MA[3][3];
    for (int i = 0; i < 3; i++) {
        MA[i][0] = M[i][1] * p2 - M[i][2] * p1;
        MA[i][1] = M[i][2] * p0 - M[i][0] * p2;
        MA[i][2] = M[i][0] * p1 - M[i][1] * p0;
    }
    /* [p]x^T M [p]x */
    float AMA[3][3];
    for (int j = 0; j < 3; j++) {
        AMA[0][j] = p2 * MA[1][j] - p1 * MA[2][j];
        AMA[1][j] = p0 * MA[2][j] - p2 * MA[0][j];
        AMA[2][j] = p1 * MA[0][j] - p0 * MA[1][j];
    }
    float Mr[3];
    for (int i = 0; i < 3; i++)
        Mr[i] = (M[i][0] * r[0] + M[i][1] * r[1]) + M[i][2] * r[2];
    float H[6][6];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            H[i][j] = AMA[i][j];
            H[i][3 + j] = -MA[j][i];
            H[3 + i][3 + j] = M[i][j];
        }
    int k = 0;
    for (int i = 0; i < 6; i++)
        for (int j = i; j < 6; j++)
            out[k++] = H[i][j];
    out[k++] = p2 * Mr[1] - p1 * Mr[2];
    out[k++] = p0 * Mr[2] - p2 * Mr[0];
    out[k++] = p1 * Mr[0] - p0 * Mr[1];
    out[k++] = -Mr[0];
    out[k++] = -Mr[1];
    out[k++] = -Mr[2];
    out[k++] = (r[0] * Mr[0] + r[1] * Mr[1]) + r[2] * Mr[2];
    for (int i = 0; i < OR_GICP_NVAL; i++)
        if (!(fabsf(out[i]) < OR_GICP_LIMIT))
            return 0;
    return 1;
}

/* Quantise a term to an integer multiple of 2^-24 (ties to even). */
int64_t or_gicp_quantise(float x)
{
    return (int64_t)llrintf(x * OR_GICP_SCALE);
}

/* Solve the 6x6 system of the quantised sums: H xi = -g by Cholesky in
 * binary64.  Returns 0 when H is not positive definite. */
int or_gicp_solve(const int64_t S[OR_GICP_NVAL], double xi[6])
{
    double H[6][6], g[6], L[6][6], y[6];
    int k = 0;
    for (int i = 0; i < 6; i++)
        for (int j = i; j < 6; j++) {
            H[i][j] = (double)S[k++] / 16777216.0;
            H[j][i] = H[i][j];
        }
    for (int i = 0; i < 6; i++)
        g[i] = (double)S[k++] / 16777216.0;
    for (int j = 0; j < 6; j++) {
        double s = H[j][j];
        for (int q = 0; q < j; q++)
            s = s - L[j][q] * L[j][q];
        if (!(s > 0.0))
            return 0;
        L[j][j] = sqrt(s);
        for (int i = j + 1; i < 6; i++) {
            double t = H[i][j];
            for (int q = 0; q < j; q++)
                t = t - L[i][q] * L[j][q];
            L[i][j] = t / L[j][j];
        }
    }
    for (int i = 0; i < 6; i++) {
        double t = -g[i];
        for (int q = 0; q < i; q++)
            t = t - L[i][q] * y[q];
        y[i] = t / L[i][i];
    }
    for (int i = 5; i >= 0; i--) {
        double t = y[i];
        for (int q = i + 1; q < 6; q++)
            t = t - L[q][i] * xi[q];
        xi[i] = t / L[i][i];
    }
    return 1;
}

/* Rotation of the quaternion (1, w/2) normalised: the rotation about w by
 * 2 atan(|w| / 2).  Row-major 3x3. */
void or_gicp_rotation(const double w[3], double R[9])
{
    double hx = w[0] * 0.5, hy = w[1] * 0.5, hz = w[2] * 0.5;
    double nrm = sqrt(((1.0 + hx * hx) + hy * hy) + hz * hz);
    double qw = 1.0 / nrm, qx = hx / nrm, qy = hy / nrm, qz = hz / nrm;
    R[0] = 1.0 - 2.0 * (qy * qy + qz * qz);
    R[1] = 2.0 * (qx * qy - qw * qz);
    R[2] = 2.0 * (qx * qz + qw * qy);
    R[3] = 2.0 * (qx * qy + qw * qz);
    R[4] = 1.0 - 2.0 * (qx * qx + qz * qz);
    R[5] = 2.0 * (qy * qz - qw * qx);
    R[6] = 2.0 * (qx * qz - qw * qy);
    R[7] = 2.0 * (qy * qz + qw * qx);
    R[8] = 1.0 - 2.0 * (qx * qx + qy * qy);
}

/* Brute-force nearest observed point of p within delta (Eq. 2's search):
 * index into the observed list (pixel order, ties to the lowest), or -1. */
static int64_t nearest_within(const float *Ixyz, int64_t nI, const float p[3], float delta2)
{
    float best = INFINITY;
    int64_t bj = -1;
    for (int64_t j = 0; j < nI; j++) {
        const float *q = Ixyz + 3 * j;
        float dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
        float d2 = (dx * dx + dy * dy) + dz * dz;
        if (d2 < best) { best = d2; bj = j; }
    }
    return (bj >= 0 && best <= delta2) ? bj : -1;
}

/* Refine n hypotheses.  poses_out (n*12) receives the refined poses, info
 * (n*2, may be NULL) the number of updates applied and the correspondences
 * of the last iteration evaluated.  Returns 0, or -2 on allocation failure. */
int or_gicp(const or_scene *sc, const or_mesh *m, int32_t label, const int32_t roi[4],
            const float *poses, int64_t n, const or_gicp_params *gp, float *poses_out,
            int32_t *info, int32_t n_threads)
{
    int64_t WH = (int64_t)sc->W * sc->H;
    float *Ixyz = malloc(sizeof(float) * 3 * (WH + 1));
    int32_t *Ipix = malloc(sizeof(int32_t) * (WH + 1));
    float *Inrm = malloc(sizeof(float) * 3 * (WH + 1));
    if (!Ixyz || !Ipix || !Inrm) {
        free(Ixyz); free(Ipix); free(Inrm);
        return -2;
    }
    int64_t nI = or_observed_points(sc, Ixyz, NULL, Ipix);
    for (int64_t j = 0; j < nI; j++)
        or_observed_normal(sc, gp->normal_jump, Ipix[j] % sc->W, Ipix[j] / sc->W, Inrm + 3 * j);
    float delta2 = sc->delta * sc->delta;
    int rc = 0;
#ifdef _OPENMP
    if (n_threads > 0)
        omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel
    {
        uint64_t *keys = malloc(sizeof(uint64_t) * WH);
        float *Rxyz = malloc(sizeof(float) * 3 * WH);
        float *Rnrm = malloc(sizeof(float) * 3 * WH);
        int32_t *Rpix = malloc(sizeof(int32_t) * WH);
        int ok = keys && Rxyz && Rnrm && Rpix;
        if (!ok) {
#pragma omp atomic write
            rc = -2;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t h = 0; h < n; h++) {
            if (!ok)
                continue;
            const float *P = poses + 12 * h;
            or_render_keys(sc, m, P, roi, keys, NULL);
            int64_t L = or_rendered_points(sc, m, P, label, keys, Rxyz, NULL, Rpix);
            for (int64_t k = 0; k < L; k++) {
                float no[3];
                or_triangle_normal(m, (int32_t)(keys[Rpix[k]] & 0xffffffffu), no);
                float *nc = Rnrm + 3 * k;
                nc[0] = (P[0] * no[0] + P[1] * no[1]) + P[2] * no[2];
                nc[1] = (P[4] * no[0] + P[5] * no[1]) + P[6] * no[2];
                nc[2] = (P[8] * no[0] + P[9] * no[1]) + P[10] * no[2];
            }
            double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, t[3] = {0, 0, 0};
            int32_t updates = 0, last_corr = 0;
            for (int32_t it = 0; it < gp->max_iters; it++) {
                float Rf[9], tf[3];
                for (int i = 0; i < 9; i++) Rf[i] = (float)R[i];
                for (int i = 0; i < 3; i++) tf[i] = (float)t[i];
                int64_t S[OR_GICP_NVAL] = {0};
                int32_t corr = 0;
                for (int64_t k = 0; k < L; k++) {
                    const float *a = Rxyz + 3 * k;
                    float p[3];
                    p[0] = ((Rf[0] * a[0] + Rf[1] * a[1]) + Rf[2] * a[2]) + tf[0];
                    p[1] = ((Rf[3] * a[0] + Rf[4] * a[1]) + Rf[5] * a[2]) + tf[1];
                    p[2] = ((Rf[6] * a[0] + Rf[7] * a[1]) + Rf[8] * a[2]) + tf[2];
                    int64_t j = nearest_within(Ixyz, nI, p, delta2);
                    if (j < 0)
                        continue;
                    float terms[OR_GICP_NVAL];
                    if (!or_gicp_terms(Rf, tf, a, Rnrm + 3 * k, Ixyz + 3 * j, Inrm + 3 * j,
                                       gp->epsilon, terms))
                        continue;
                    for (int i = 0; i < OR_GICP_NVAL; i++)
                        S[i] += or_gicp_quantise(terms[i]);
                    corr++;
                }
                last_corr = corr;
                double xi[6];
                if (corr < gp->min_corr || !or_gicp_solve(S, xi))
                    break;
                double dR[9], R2[9], t2[3];
                or_gicp_rotation(xi, dR);
                for (int i = 0; i < 3; i++) {
                    for (int j = 0; j < 3; j++)
                        R2[3 * i + j] = (dR[3 * i] * R[j] + dR[3 * i + 1] * R[3 + j]) + dR[3 * i + 2] * R[6 + j];
                    t2[i] = ((dR[3 * i] * t[0] + dR[3 * i + 1] * t[1]) + dR[3 * i + 2] * t[2]) + xi[3 + i];
                }
                memcpy(R, R2, sizeof(R));
                memcpy(t, t2, sizeof(t));
                updates++;
                double sr = (double)gp->stop_rot, st = (double)gp->stop_trans;
                if ((xi[0] * xi[0] + xi[1] * xi[1]) + xi[2] * xi[2] < sr * sr &&
                    (xi[3] * xi[3] + xi[4] * xi[4]) + xi[5] * xi[5] < st * st)
                    break;
            }
            /* refined pose = increment o input pose */
            float *Q = poses_out + 12 * h;
            for (int i = 0; i < 3; i++) {
                for (int j = 0; j < 3; j++)
                    Q[4 * i + j] = (float)((R[3 * i] * (double)P[j] + R[3 * i + 1] * (double)P[4 + j])
                                           + R[3 * i + 2] * (double)P[8 + j]);
                Q[4 * i + 3] = (float)(((R[3 * i] * (double)P[3] + R[3 * i + 1] * (double)P[7])
                                        + R[3 * i + 2] * (double)P[11]) + t[i]);
            }
            if (info) {
                info[2 * h] = updates;
                info[2 * h + 1] = last_corr;
            }
        }
        free(keys); free(Rxyz); free(Rnrm); free(Rpix);
    }
    free(Ixyz); free(Ipix); free(Inrm);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Monotone Scene Generation tree (Sec. III, Fig. 2; variant 2.0-B)        */
/* ---------------------------------------------------------------------- */
/*
 * A state holds the objects placed so far as three per-pixel images:
 *   depth  nearest rendered depth of the placed objects on the stride
 *          lattice (0.1 mm, 0 = none): the composed rendered scene;
 *   mark   observed pixels found as the nearest neighbour of an explained
 *          rendered point of a placed object;
 *   vol    observed pixels inside a placed object's admissible volume V
 *          (already counted in J_o).
 * Adding object O at pose h is an edge of the tree.  The edge is refused
 * (costs -1, -1) when O occludes a placed object: some lattice pixel where O
 * renders at depth d with state depth s > 0 and d + m < s (m = the occluder
 * margin, or 0 when occluder marking is off).  Otherwise O's point cloud
 * Delta R is its rendered lattice pixels not behind the state (s == 0 or
 * d < s) and not behind the observed depth (the usual occluder rule), and
 *   dJ_r = points of Delta R that are not explained (Eq. 2, Eq. 4),
 *   dJ_o = observed points in V(O) \ vol that are marked neither in the
 *          state nor by Delta R (Eq. 1 over the newly covered volume).
 * The child state is the parent with O's visible lattice pixels composed
 * into depth, Delta R's marks added to mark and V(O) added to vol.
 * Readings: the occlusion test and the composition use the stride lattice;
 * J_o uses the nearest-neighbour marks (jo_mode 0).
 */
int or_score_tree(const or_scene *sc, const or_mesh *m, int32_t label, const int32_t roi[4],
                  const float *poses, int64_t n, const uint32_t *p_depth, const uint8_t *p_mark,
                  const uint8_t *p_vol, int32_t *costs, int32_t *band, uint32_t *c_depth,
                  uint8_t *c_mark, uint8_t *c_vol, int32_t n_threads)
{
    int64_t WH = (int64_t)sc->W * sc->H;
    int64_t s = sc->stride;
    int32_t margin = sc->occ_margin > 0 ? sc->occ_margin : 0;
    float *Ixyz = malloc(sizeof(float) * 3 * (WH + 1));
    float *Ilab = malloc(sizeof(float) * 3 * (WH + 1));
    int32_t *Ipix = malloc(sizeof(int32_t) * (WH + 1));
    if (!Ixyz || !Ilab || !Ipix) {
        free(Ixyz); free(Ilab); free(Ipix);
        return -2;
    }
    int64_t nI = or_observed_points(sc, Ixyz, Ilab, Ipix);
    float delta2 = sc->delta * sc->delta;
    int write_child = c_depth && c_mark && c_vol && n == 1;
    if (write_child) {
        memcpy(c_depth, p_depth, sizeof(uint32_t) * WH);
        memcpy(c_mark, p_mark, WH);
        memcpy(c_vol, p_vol, WH);
    }
    int rc = 0;
#ifdef _OPENMP
    if (n_threads > 0)
        omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel
    {
        uint64_t *keys = malloc(sizeof(uint64_t) * WH);
        float *Rxyz = malloc(sizeof(float) * 3 * WH);
        uint8_t *Rrgb = malloc(3 * WH);
        int32_t *Rpix = malloc(sizeof(int32_t) * WH);
        uint8_t *mark = malloc(nI + 1);
        int ok = keys && Rxyz && Rrgb && Rpix && mark;
        if (!ok) {
#pragma omp atomic write
            rc = -2;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t h = 0; h < n; h++) {
            if (!ok)
                continue;
            const float *P = poses + 12 * h;
            or_render_keys(sc, m, P, roi, keys, NULL);
            /* monotone test and composition over the rendered lattice pixels */
            int occludes = 0;
            for (int64_t i = 0; i < WH && !occludes; i++) {
                int64_t u = i % sc->W, v = i / sc->W;
                if (keys[i] == OR_EMPTY || u % s != 0 || v % s != 0)
                    continue;
                int64_t d = (int64_t)(keys[i] >> 32), sd = p_depth[i];
                if (sd > 0 && d + margin < sd)
                    occludes = 1;
            }
            if (occludes) {
                costs[2 * h] = -1;
                costs[2 * h + 1] = -1;
                if (band) band[h] = 0;
                continue;
            }
            int64_t L = or_rendered_points(sc, m, P, label, keys, Rxyz, Rrgb, Rpix);
            memset(mark, 0, nI + 1);
            int32_t Jr = 0, nband = 0;
            for (int64_t k = 0; k < L; k++) {
                int64_t i = Rpix[k];
                int64_t d = (int64_t)(keys[i] >> 32), sd = p_depth[i];
                if (sd > 0 && !(d < sd))
                    continue;                       /* behind a placed object */
                const float *q = Rxyz + 3 * k;
                float best = INFINITY;
                int64_t bj = -1;
                for (int64_t j = 0; j < nI; j++) {
                    const float *p = Ixyz + 3 * j;
                    float dx = q[0] - p[0], dy = q[1] - p[1], dz = q[2] - p[2];
                    float d2 = (dx * dx + dy * dy) + dz * dz;
                    if (d2 < best) { best = d2; bj = j; }
                }
                int explained = bj >= 0 && best <= delta2;
                if (explained && sc->color_check) {
                    float lq[3], gap;
                    or_srgb_to_lab(Rrgb + 3 * k, lq);
                    float dE = or_ciede2000(lq, Ilab + 3 * bj, &gap);
                    if (fabsf(dE - sc->tau_c) <= 1e-3f || gap <= 1e-3f)
                        nband++;
                    if (dE > sc->tau_c)
                        explained = 0;
                }
                if (explained)
                    mark[bj] = 1;
                else
                    Jr++;
            }
            int32_t Jo = 0;
            for (int64_t j = 0; j < nI; j++) {
                int64_t i = Ipix[j];
                if (p_vol[i] || !in_volume(sc, m, P, label, roi, i, Ixyz + 3 * j))
                    continue;
                if (!mark[j] && !p_mark[i])
                    Jo++;
            }
            costs[2 * h] = Jo;
            costs[2 * h + 1] = Jr;
            if (band) band[h] = nband;
            if (write_child) {
                for (int64_t i = 0; i < WH; i++) {
                    int64_t u = i % sc->W, v = i / sc->W;
                    if (keys[i] == OR_EMPTY || u % s != 0 || v % s != 0)
                        continue;
                    uint32_t d = (uint32_t)(keys[i] >> 32);
                    if (p_depth[i] == 0 || d < p_depth[i])
                        c_depth[i] = d;
                }
                for (int64_t j = 0; j < nI; j++) {
                    if (mark[j])
                        c_mark[Ipix[j]] = 1;
                    if (in_volume(sc, m, P, label, roi, Ipix[j], Ixyz + 3 * j))
                        c_vol[Ipix[j]] = 1;
                }
            }
        }
        free(keys); free(Rxyz); free(Rrgb); free(Rpix); free(mark);
    }
    free(Ixyz); free(Ilab); free(Ipix);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* ADD and ADD-S pose errors (the accuracy measure of Sec. VI)             */
/* ---------------------------------------------------------------------- */

/* Mean over the model points x of the distance between x under pose A and
 * (symmetric: the closest model point, else the same point) under pose B,
 * in binary64 (poses row-major 3x4). */
double or_add_s(const float *verts, int32_t n_verts, const float A[12], const float B[12], int32_t symmetric)
{
    if (n_verts < 1)
        return 0.0;
    double *pb = malloc(sizeof(double) * 3 * n_verts);
    if (!pb)
        return -1.0;
    for (int32_t i = 0; i < n_verts; i++) {
        const float *x = verts + 3 * i;
        for (int r = 0; r < 3; r++)
            pb[3 * i + r] = (double)B[4 * r] * x[0] + (double)B[4 * r + 1] * x[1] + (double)B[4 * r + 2] * x[2]
                            + (double)B[4 * r + 3];
    }
    double sum = 0.0;
    for (int32_t i = 0; i < n_verts; i++) {
        const float *x = verts + 3 * i;
        double pa[3];
        for (int r = 0; r < 3; r++)
            pa[r] = (double)A[4 * r] * x[0] + (double)A[4 * r + 1] * x[1] + (double)A[4 * r + 2] * x[2]
                    + (double)A[4 * r + 3];
        double best;
        if (symmetric) {
            best = INFINITY;
            for (int32_t j = 0; j < n_verts; j++) {
                double dx = pa[0] - pb[3 * j], dy = pa[1] - pb[3 * j + 1], dz = pa[2] - pb[3 * j + 2];
                double d2 = dx * dx + dy * dy + dz * dz;
                if (d2 < best)
                    best = d2;
            }
        } else {
            double dx = pa[0] - pb[3 * i], dy = pa[1] - pb[3 * i + 1], dz = pa[2] - pb[3 * i + 2];
            best = dx * dx + dy * dy + dz * dz;
        }
        sum += sqrt(best);
    }
    free(pb);
    return sum / n_verts;
}

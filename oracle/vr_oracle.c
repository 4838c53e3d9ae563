/*
 * vr_oracle.c -- plain, slow, FP64 CPU ray caster for noisy spectral cubes.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this library.  It shares no code, header, table
 * or helper with the CUDA path; it reads the cube in its plain linear layout
 * (x fastest, then y, then z) and knows nothing of bricks.
 *
 * What it computes (paper §3.1, process item 3: every output pixel becomes
 * one ray, and the ray is mapped to RGBA by a pre-selected transfer
 * function; the abstract's emphasis on low signal-to-noise data motivates
 * the clip).  The paper prints no formulas, so each step below is the
 * reading this project fixes, evaluated in double precision on the stored
 * voxel values:
 *
 *   camera -> ray   u = px + 1/2 - w/2, v = py + 1/2 - h/2;
 *                   ortho: o = eye + u du + v dv, d = fwd / |fwd|;
 *                   persp: o = eye, d = (fwd + u du + v dv) / |...|.
 *   ray / box       box = [0, n-1] per axis (between the first and last voxel
 *                   centres).  Slab test; an axis with d_i == 0 passes iff
 *                   0 <= o_i <= n_i - 1 (no division).  t_entry = max(0,
 *                   max t_near), t_exit = min t_far, hit iff t_exit >= t_entry.
 *   samples         K = floor((t_exit - t_entry) / step) + 1 if hit, else 0;
 *                   t_k = t_entry + k step from the integer k; p_k = o + t_k d
 *                   clamped to the box.
 *   trilinear       i0 = min(floor(p), n - 2), f = p - i0 per axis; the eight
 *                   corners are interpolated along x, then y, then z with
 *                   lerp(a, b, f) = a + f (b - a).
 *   transfer fn.    s < clip: fully transparent (skipped).  Otherwise
 *                   x = clamp((s - v_lo) / (v_hi - v_lo), 0, 1) (N - 1),
 *                   i = min(floor(x), N - 2), RGBA = lerp(L'[i], L'[i+1], x - i)
 *                   where L' is the table with alpha' = 1 - (1 - alpha)^step
 *                   (opacity per unit voxel length corrected to the step).
 *   composite       front to back: C += (1 - A) alpha rgb, A += (1 - A) alpha;
 *                   after each composited sample the ray stops once
 *                   A >= term_alpha.  Output premultiplied (C, A); K = 0 -> 0.
 *   MIP             max_k s_k (raw value); K = 0 -> -infinity.
 *   SUM             sum_k s_k * step (an additive mode used only by tests).
 *
 * Storage types: float32 values; IEEE binary16 bit patterns (decoded here
 * from the format's definition); int8 codes q with a per-frequency-plane
 * scale and offset, value = q * scale[z] + offset[z] evaluated in double.
 *
 * Acceptance sets.  Three places turn an arbitrarily small perturbation of
 * the arithmetic into a finite change of the result: the sample count K, the
 * clip test, and the termination test.  A single-precision implementation can
 * legitimately land on the other side of each.  For every pixel the oracle
 * therefore returns the primary double-precision result plus the results of
 * the alternative decisions whose deciding quantity lies within a stated band
 * of its threshold.  The bands are inputs (the tests state them) and model
 * the rounding of a single-precision evaluation of the same definition:
 *   band_t      relative error of a ray parameter t per unit |t| (division,
 *               subtraction, the direction's rounding);
 *   band_pos    absolute error of the ray origin (orthographic origins are
 *               computed from the camera), per coordinate;
 *   band_clip   relative error of an interpolated value, per unit of its
 *               largest |corner|;
 *   band_k      an absolute floor of the K band;
 *   band_a      the termination band in alpha.
 * From them, per ray:  a slab parameter t decided by axis a is uncertain by
 *   e(t) = (band_t |t| + band_pos) / |d_a|
 * (t_entry is exact when the camera is inside the box, t_entry = 0), and per
 * sample k the position by
 *   e_p  = e(t_entry) + band_t (|t_k| + max|o| + max|p_k|) + band_pos.
 *   K band      (t_exit - t_entry)/step within band_k + (e(t_entry) +
 *               e(t_exit))/step of an integer (this also covers near-miss /
 *               grazing rays, K = 0 <-> 1, and rays lying within band_pos of
 *               a face plane they are parallel to);
 *   clip band   |s - clip| <= band_clip max(1, max|corner|) + e_p |grad s|_1
 *               where the table's alpha at the clip level is non-zero (the
 *               sample's decision is flipped alone; |grad s|_1 is the sum of
 *               the trilinear field's partial derivatives' magnitudes there);
 *   term band   every composited sample from the first with A >= ta - band_a
 *               up to the first with A >= ta + band_a is a possible stop.
 * Flags: bit 0 K tie, bit 1 clip tie, bit 2 termination tie, bit 3 the
 * alternative list was truncated at VRO_MAXALT (or more clip ties than
 * VRO_MAXCLIP were found).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define VRO_MAXALT 16
#define VRO_MAXCLIP 4

enum { VRO_F32 = 0, VRO_F16 = 1, VRO_I8 = 2 };
enum { VRO_MIP = 0, VRO_COMPOSITE = 1, VRO_SUM = 2 };
enum { VRO_ORTHO = 0, VRO_PERSP = 1 };

/* One camera record as laid out in memory by the callers (64 bytes). */
typedef struct {
    int32_t proj;
    float eye[3], fwd[3], du[3], dv[3], pad[3];
} vro_camera;

typedef struct {
    int64_t n[3];          /* nx, ny, nz */
    int32_t dtype;         /* VRO_F32 / VRO_F16 / VRO_I8 */
    const void* data;      /* n[0]*n[1]*n[2] elements, x fastest */
    const float* scale;    /* int8 only: per z plane */
    const float* offset;   /* int8 only: per z plane */
} vro_volume;

typedef struct {
    const float* lut;      /* n_lut x 4 (r, g, b, alpha per unit length) */
    int32_t n_lut;
    double v_lo, v_hi, clip, term_alpha;
} vro_tf;

typedef struct {
    double band_k, band_pos, band_clip, band_a, band_t;
} vro_bands;

/* ------------------------------------------------------------------ */
/* storage decoding                                                     */
/* ------------------------------------------------------------------ */

/* IEEE 754 binary16: 1 sign bit, 5 exponent bits (bias 15), 10 fraction bits. */
static double half_to_double(uint16_t h)
{
    int sign = (h >> 15) & 1;
    int e = (h >> 10) & 0x1f;
    int m = h & 0x3ff;
    double v;
    if (e == 0)
        v = ldexp((double)m, -24);                 /* zero / subnormal */
    else if (e == 31)
        v = (m == 0) ? INFINITY : NAN;
    else
        v = ldexp((double)(1024 + m), e - 25);     /* (1 + m/1024) 2^(e-15) */
    return sign ? -v : v;
}

static double voxel(const vro_volume* vol, int64_t i, int64_t j, int64_t k)
{
    int64_t idx = (k * vol->n[1] + j) * vol->n[0] + i;
    switch (vol->dtype) {
    case VRO_F32:
        return (double)((const float*)vol->data)[idx];
    case VRO_F16:
        return half_to_double(((const uint16_t*)vol->data)[idx]);
    default:
        return (double)((const int8_t*)vol->data)[idx] * (double)vol->scale[k]
               + (double)vol->offset[k];
    }
}

/* ------------------------------------------------------------------ */
/* geometry                                                             */
/* ------------------------------------------------------------------ */

static void make_ray(const vro_camera* c, int w, int h, int px, int py,
                     double o[3], double d[3])
{
    double u = px + 0.5 - w / 2.0;
    double v = py + 0.5 - h / 2.0;
    double nrm = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (c->proj == VRO_ORTHO) {
            o[a] = (double)c->eye[a] + u * (double)c->du[a] + v * (double)c->dv[a];
            d[a] = (double)c->fwd[a];
        } else {
            o[a] = (double)c->eye[a];
            d[a] = (double)c->fwd[a] + u * (double)c->du[a] + v * (double)c->dv[a];
        }
        nrm += d[a] * d[a];
    }
    nrm = sqrt(nrm);
    for (int a = 0; a < 3; ++a) d[a] /= nrm;
}

/* Slab test over the axes the ray is not parallel to: t_near/t_far (t_near
 * unclamped).  For the parallel axes (d_i == 0, no division) it reports
 * *miss_dist, how far outside [0, n_i - 1] the worst excluded coordinate lies
 * (0 when none is excluded), and *face_dist, the smallest distance of an
 * included coordinate to one of its two face planes (infinity if none).
 * *dn and *df are |d_a| of the axes that decide t_near and t_far.          */
static void slab(const double o[3], const double d[3], const int64_t n[3],
                 double* t_near, double* t_far, double* miss_dist, double* face_dist,
                 double* dn, double* df)
{
    double tn = -INFINITY, tf = INFINITY;
    *dn = 1.0;
    *df = 1.0;
    *miss_dist = 0.0;
    *face_dist = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double hi = (double)(n[a] - 1);
        if (d[a] != 0.0) {
            double ta = (0.0 - o[a]) / d[a];
            double tb = (hi - o[a]) / d[a];
            double lo_t = ta < tb ? ta : tb;
            double hi_t = ta < tb ? tb : ta;
            if (lo_t > tn) { tn = lo_t; *dn = fabs(d[a]); }
            if (hi_t < tf) { tf = hi_t; *df = fabs(d[a]); }
        } else if (o[a] < 0.0 || o[a] > hi) {
            double md = o[a] < 0.0 ? -o[a] : o[a] - hi;
            if (md > *miss_dist) *miss_dist = md;
        } else {
            double fd = fmin(o[a], hi - o[a]);
            if (fd < *face_dist) *face_dist = fd;
        }
    }
    *t_near = tn;
    *t_far = tf;
}

static double lerp(double a, double b, double f) { return a + f * (b - a); }

/* One trilinear sample at o + t d.  When sens is not NULL it receives what
 * the clip band needs: sens[0] the sum of the magnitudes of the field's
 * partial derivatives at the point (per unit length), sens[1] the largest
 * |corner|, sens[2] the largest |coordinate| of the (unclamped) position.  */
static double sample_sens(const vro_volume* vol, const double o[3], const double d[3],
                          double t, double* sens)
{
    double p[3], f[3];
    int64_t i0[3];
    for (int a = 0; a < 3; ++a) {
        double hi = (double)(vol->n[a] - 1);
        p[a] = o[a] + t * d[a];
        if (p[a] < 0.0) p[a] = 0.0;
        if (p[a] > hi) p[a] = hi;
        int64_t fl = (int64_t)floor(p[a]);
        if (fl > vol->n[a] - 2) fl = vol->n[a] - 2;
        i0[a] = fl;
        f[a] = p[a] - (double)fl;
    }
    double c[2][2][2];
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx)
                c[cz][cy][cx] = voxel(vol, i0[0] + cx, i0[1] + cy, i0[2] + cz);
    double y0z0 = lerp(c[0][0][0], c[0][0][1], f[0]);
    double y1z0 = lerp(c[0][1][0], c[0][1][1], f[0]);
    double y0z1 = lerp(c[1][0][0], c[1][0][1], f[0]);
    double y1z1 = lerp(c[1][1][0], c[1][1][1], f[0]);
    double z0 = lerp(y0z0, y1z0, f[1]);
    double z1 = lerp(y0z1, y1z1, f[1]);
    if (sens) {
        double gx = lerp(lerp(c[0][0][1] - c[0][0][0], c[0][1][1] - c[0][1][0], f[1]),
                         lerp(c[1][0][1] - c[1][0][0], c[1][1][1] - c[1][1][0], f[1]), f[2]);
        double gy = lerp(y1z0 - y0z0, y1z1 - y0z1, f[2]);
        double gz = z1 - z0;
        double cm = 0.0, pm = 0.0;
        for (int cz = 0; cz < 2; ++cz)
            for (int cy = 0; cy < 2; ++cy)
                for (int cx = 0; cx < 2; ++cx) cm = fmax(cm, fabs(c[cz][cy][cx]));
        for (int a = 0; a < 3; ++a) pm = fmax(pm, fabs(o[a] + t * d[a]));
        sens[0] = fabs(gx) + fabs(gy) + fabs(gz);
        sens[1] = cm;
        sens[2] = pm;
    }
    return lerp(z0, z1, f[2]);
}

static double sample(const vro_volume* vol, const double o[3], const double d[3],
                     double t)
{
    return sample_sens(vol, o, d, t, NULL);
}

/* ------------------------------------------------------------------ */
/* rounding bands of one ray                                            */
/* ------------------------------------------------------------------ */

/* What a single-precision evaluation of the ray may get wrong (see the
 * header): e_te, the error of t_entry; omax, max |o_i|.  */
typedef struct {
    double e_te, omax;
} ray_err;

/* Error of a slab parameter t decided by an axis with |d_a| = da.        */
static double t_err(const vro_bands* b, double t, double da)
{
    return (b->band_t * fabs(t) + b->band_pos) / da;
}

static ray_err make_ray_err(const vro_bands* b, const double o[3], double tn, double dn)
{
    ray_err e;
    double et = isfinite(tn) ? t_err(b, tn, dn) : 0.0;
    e.e_te = tn > -et ? et : 0.0;     /* t_entry = 0 exactly when the camera is inside */
    e.omax = fmax(fabs(o[0]), fmax(fabs(o[1]), fabs(o[2])));
    return e;
}

/* Position error of the sample at t (see the header).                  */
static double pos_err(const vro_bands* b, const ray_err* e, double t, double pmax)
{
    return e->e_te + b->band_t * (fabs(t) + e->omax + pmax) + b->band_pos;
}

/* May a single-precision evaluation put this sample on the other side of
 * the clip?                                                              */
static int clip_tie(const vro_bands* b, const ray_err* e, const vro_tf* tf, double s,
                    double t, const double sens[3])
{
    double band = b->band_clip * fmax(1.0, sens[1]) + pos_err(b, e, t, sens[2]) * sens[0];
    return fabs(s - tf->clip) <= band;
}

/* ------------------------------------------------------------------ */
/* transfer function                                                    */
/* ------------------------------------------------------------------ */

/* Table with alpha corrected from unit voxel length to the step length. */
static void correct_table(const vro_tf* tf, double step, double* lutc)
{
    for (int i = 0; i < tf->n_lut; ++i) {
        for (int c = 0; c < 3; ++c) lutc[4 * i + c] = (double)tf->lut[4 * i + c];
        double a = (double)tf->lut[4 * i + 3];
        lutc[4 * i + 3] = 1.0 - pow(1.0 - a, step);
    }
}

static void classify(const vro_tf* tf, const double* lutc, double s, double rgba[4])
{
    int n = tf->n_lut;
    double x = (s - tf->v_lo) / (tf->v_hi - tf->v_lo);
    if (x < 0.0) x = 0.0;
    if (x > 1.0) x = 1.0;
    x *= (double)(n - 1);
    int i = (int)floor(x);
    if (i > n - 2) i = n - 2;
    double w = x - (double)i;
    for (int c = 0; c < 4; ++c) rgba[c] = lerp(lutc[4 * i + c], lutc[4 * (i + 1) + c], w);
}

/* ------------------------------------------------------------------ */
/* per-ray marches                                                      */
/* ------------------------------------------------------------------ */

typedef struct {
    double v[VRO_MAXALT][4];
    int n;
    int flags;
} alts;

static void push(alts* r, const double v[4])
{
    for (int i = 0; i < r->n; ++i)      /* identical results add nothing */
        if (r->v[i][0] == v[0] && r->v[i][1] == v[1] && r->v[i][2] == v[2] &&
            r->v[i][3] == v[3])
            return;
    if (r->n >= VRO_MAXALT) { r->flags |= 8; return; }
    memcpy(r->v[r->n++], v, 4 * sizeof(double));
}

/* MIP or SUM over samples 0..K-1; returns the count of samples. */
static int64_t march_scalar(const vro_volume* vol, int mode, const double o[3],
                            const double d[3], double t_entry, int64_t K, double step,
                            double* result)
{
    double m = -INFINITY, acc = 0.0;
    for (int64_t k = 0; k < K; ++k) {
        double s = sample(vol, o, d, t_entry + (double)k * step);
        if (mode == VRO_MIP) { if (s > m) m = s; }
        else acc += s * step;
    }
    *result = (mode == VRO_MIP) ? m : acc;
    return K;
}

/* Emission-absorption march over samples 0..K-1.  flip_k >= 0 inverts the
 * clip decision of that one sample.  The primary stopping state is pushed to
 * *r first, then every other possible stopping state of the term band.  When
 * more than VRO_MAXALT - 1 band states occur, the first VRO_MAXALT - 1 and the
 * latest are kept (flag 8); all states in a band lie between those, because
 * C and A never decrease.  Samples near the clip are reported through
 * clip_k[] (up to VRO_MAXCLIP).  Returns the primary rule's sample count. */
static int64_t march_composite(const vro_volume* vol, const vro_tf* tf,
                               const double* lutc, const double o[3], const double d[3],
                               double t_entry, int64_t K, double step, int64_t flip_k,
                               const vro_bands* b, const ray_err* e, alts* r,
                               int64_t* clip_k, int* n_clip)
{
    double C[3] = {0, 0, 0}, A = 0.0;
    double ta = tf->term_alpha;
    double clip_rgba[4];
    classify(tf, lutc, tf->clip, clip_rgba);
    double prim[4];
    int have_prim = 0;
    int64_t prim_count = K;
    double cand[VRO_MAXALT][4];
    int n_cand = 0;
    if (n_clip) *n_clip = 0;
    for (int64_t k = 0; k < K; ++k) {
        double t = t_entry + (double)k * step, sens[3];
        double s = sample_sens(vol, o, d, t, sens);
        int keep = !(s < tf->clip);
        if (n_clip && clip_rgba[3] > 0.0 && clip_tie(b, e, tf, s, t, sens)) {
            if (*n_clip < VRO_MAXCLIP)
                clip_k[(*n_clip)++] = k;
            else
                r->flags |= 8;
        }
        if (k == flip_k) keep = !keep;
        if (!keep) continue;
        double rgba[4];
        classify(tf, lutc, s, rgba);
        double wgt = (1.0 - A) * rgba[3];
        for (int c = 0; c < 3; ++c) C[c] += wgt * rgba[c];
        A += wgt;
        if (A >= ta - b->band_a) {
            double st[4] = {C[0], C[1], C[2], A};
            int slot;
            if (n_cand < VRO_MAXALT) {
                slot = n_cand++;
            } else {
                slot = VRO_MAXALT - 1;
                r->flags |= 8;
            }
            memcpy(cand[slot], st, sizeof st);
            if (!have_prim && A >= ta) {
                memcpy(prim, st, sizeof st);
                have_prim = 1;
                prim_count = k + 1;
            }
            if (A >= ta + b->band_a) break;
        }
    }
    if (!have_prim) {             /* never reached the threshold: end state */
        prim[0] = C[0]; prim[1] = C[1]; prim[2] = C[2]; prim[3] = A;
        prim_count = K;
    }
    int before = r->n;
    push(r, prim);
    for (int i = 0; i < n_cand; ++i) push(r, cand[i]);
    if (r->n - before > 1) r->flags |= 4;
    return prim_count;
}

/* ------------------------------------------------------------------ */
/* one pixel                                                            */
/* ------------------------------------------------------------------ */

static void render_pixel(const vro_volume* vol, const vro_camera* cam, int w, int h,
                         int px, int py, int mode, double step, const vro_tf* tf,
                         const double* lutc, const vro_bands* b, alts* r,
                         int64_t* nsamples)
{
    double o[3], d[3];
    make_ray(cam, w, h, px, py, o, d);

    double tn, tf_, miss_dist, face_dist, dn, df;
    slab(o, d, vol->n, &tn, &tf_, &miss_dist, &face_dist, &dn, &df);
    double t_entry = tn > 0.0 ? tn : 0.0;
    double t_exit = tf_;
    double q = (t_exit - t_entry) / step;
    int hit = miss_dist == 0.0 && t_exit >= t_entry;
    ray_err e = make_ray_err(b, o, tn, dn);
    double wq = b->band_k + (e.e_te + t_err(b, t_exit, df)) / step;

    /* candidate sample counts, primary first */
    int64_t Ks[4];
    int nK = 0;
    if (hit) {
        double fl = floor(q);
        int64_t K = (int64_t)fl + 1;
        Ks[nK++] = K;
        if (q - fl < wq) Ks[nK++] = K - 1;
        if (q - fl > 1.0 - wq) Ks[nK++] = K + 1;
        if (face_dist <= b->band_pos) Ks[nK++] = 0;
    } else {
        Ks[nK++] = 0;
        /* a near miss: slightly different rounding could give a short hit */
        if (miss_dist <= b->band_pos && q >= -wq)
            Ks[nK++] = q < 0.0 ? 1 : (int64_t)floor(q) + 1;
    }
    if (nK > 1) r->flags |= 1;

    for (int ik = 0; ik < nK; ++ik) {
        int64_t K = Ks[ik];
        if (mode == VRO_COMPOSITE) {
            if (K == 0) {
                double z[4] = {0, 0, 0, 0};
                push(r, z);
                if (ik == 0) *nsamples = 0;
                continue;
            }
            int64_t clip_k[VRO_MAXCLIP];
            int n_clip = 0;
            int64_t cnt = march_composite(vol, tf, lutc, o, d, t_entry, K, step, -1, b, &e,
                                          r, clip_k, &n_clip);
            if (ik == 0) *nsamples = cnt;
            for (int ic = 0; ic < n_clip; ++ic) {
                r->flags |= 2;
                march_composite(vol, tf, lutc, o, d, t_entry, K, step, clip_k[ic], b, &e, r,
                                NULL, NULL);
            }
        } else {
            double v[4] = {0, 0, 0, 0};
            int64_t cnt = march_scalar(vol, mode, o, d, t_entry, K, step, &v[0]);
            push(r, v);
            if (ik == 0) *nsamples = cnt;
        }
    }
}

/* ------------------------------------------------------------------ */
/* exported entry points                                                */
/* ------------------------------------------------------------------ */

int vro_maxalt(void) { return VRO_MAXALT; }

int vro_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Render a list of pixels.  pix holds npix triples (view, px, py).  For pixel
 * i, out[i*VRO_MAXALT*4 + a*4 + c] is channel c of acceptable result a
 * (a < nalt[i]; a = 0 is the primary double-precision result; MIP and SUM use
 * channel 0 only).  nsamples[i] is the primary result's count of evaluated
 * samples.  nthreads <= 0 uses the OpenMP default.  Returns 0, or -1 on bad
 * arguments.
 */
int vro_render(const vro_volume* vol, const vro_camera* cams, int n_views, int w, int h,
               int mode, double step, const vro_tf* tf, const vro_bands* bands,
               const int32_t* pix, int64_t npix, double* out, int32_t* nalt,
               int32_t* flags, int64_t* nsamples, int nthreads)
{
    if (!vol || !cams || !tf || !bands || !pix || !out || !nalt || !flags || !nsamples)
        return -1;
    if (vol->n[0] < 2 || vol->n[1] < 2 || vol->n[2] < 2 || !(step > 0.0) ||
        tf->n_lut < 2 || w <= 0 || h <= 0 || n_views <= 0)
        return -1;
    if (mode != VRO_MIP && mode != VRO_COMPOSITE && mode != VRO_SUM) return -1;
    double* lutc = (double*)malloc(sizeof(double) * 4 * (size_t)tf->n_lut);
    if (!lutc) return -1;
    correct_table(tf, step, lutc);
    int bad = 0;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt) reduction(| : bad)
#endif
    for (int64_t i = 0; i < npix; ++i) {
        int view = pix[3 * i], px = pix[3 * i + 1], py = pix[3 * i + 2];
        if (view < 0 || view >= n_views || px < 0 || px >= w || py < 0 || py >= h) {
            bad = 1;
            continue;
        }
        alts r;
        r.n = 0;
        r.flags = 0;
        int64_t ns = 0;
        render_pixel(vol, &cams[view], w, h, px, py, mode, step, tf, lutc, bands, &r, &ns);
        memset(&out[i * VRO_MAXALT * 4], 0, sizeof(double) * VRO_MAXALT * 4);
        for (int a = 0; a < r.n; ++a)
            memcpy(&out[(i * VRO_MAXALT + a) * 4], r.v[a], 4 * sizeof(double));
        nalt[i] = r.n;
        flags[i] = r.flags;
        nsamples[i] = ns;
    }
    (void)nthreads;
    free(lutc);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* sub-cubes rendered independently, then integrated                    */
/* ------------------------------------------------------------------ */

/*
 * The paper's pipeline splits the cube into sub-cubes, renders each into its
 * own partial image and combines the partial images (§3.1 items 1, 4, 5;
 * the garbled "scene integration" sentence is read as combining the partial
 * images by the compositing operator in visibility order).  Here sub-cube i
 * owns the cells [cell_lo[i], cell_lo[i+1]) along z (the last one up to
 * n_z - 1); a sample belongs to the sub-cube of its cell, floor(z) of its
 * position before clamping (the first sub-cube also takes heights below 0,
 * the last those above).  Each sub-cube's partial result starts empty and
 * sees only its own samples, in the ray's order; a composite partial stops
 * once its own alpha reaches term_alpha.  The partial results are combined
 * in the order the ray meets the sub-cubes: "over" for composite,
 *   C += (1 - A) C_i,  A += (1 - A) A_i,
 * max for MIP, addition for SUM.  Without termination this is the one-pass
 * result (the operator is associative); with it, a ray may pass an opaque
 * sub-cube's partial and keep contributions behind it, attenuated.
 * Acceptance set as for vro_render: the primary FP64 result plus the results
 * of single decisions changed within the bands -- K - 1 or K + 1 (K band), one
 * sample's clip decision inverted (clip band), one sample given to the
 * sub-cube on the other side of a boundary plane it lies within rounding of
 * (the position band), one sub-cube's partial stopped at another sample of
 * its termination band.  Flags: bit 0 K tie, bit 1 clip tie, bit 2
 * termination tie, bit 3 truncated (more ties than the lists hold), bit 4 a
 * sample within rounding of a sub-cube boundary plane.
 */
#define VRO_MAXMOVE 4
#define VRO_MAXSTOP 8

static int segment_of(double z, const int64_t* cell_lo, int n_sub)
{
    double c = floor(z);
    int i = 0;
    while (i + 1 < n_sub && c >= (double)cell_lo[i + 1]) ++i;
    return i;
}

/* One decision of a sub-cube march changed from the primary rule.        */
typedef struct {
    int64_t flip_k;        /* this sample's clip decision inverted (-1: none) */
    int64_t move_k;        /* this sample belongs to sub-cube move_to (-1: none) */
    int move_to;
    int stop_seg;          /* sub-cube stop_seg stops after composited sample stop_k */
    int64_t stop_k;        /* (-1: every sub-cube stops by the threshold)          */
} sub_variant;

/* The ties a probing march finds.                                       */
typedef struct {
    int64_t clip_k[VRO_MAXCLIP];
    int n_clip;
    int64_t move_k[VRO_MAXMOVE];
    int move_to[VRO_MAXMOVE];
    int n_move;
    int stop_seg[VRO_MAXSTOP];
    int64_t stop_k[VRO_MAXSTOP];
    int n_stop;
    int flags;
} sub_ties;

typedef struct {
    double *C, *A, *V;
    int *done, *order;
} sub_work;

/* March samples 0..K-1 of a ray as n_sub independent partials and combine
 * them in the ray's order into res.  With ties != NULL the march probes:
 * every sub-cube composites on until its alpha reaches term_alpha + band_a,
 * and the ties met on the way are listed (res is then not the result).   */
static void subcube_march(const vro_volume* vol, const double o[3], const double d[3],
                          double t_entry, int64_t K, double step, int mode,
                          const vro_tf* tf, const double* lutc, double clip_alpha,
                          const vro_bands* b, const ray_err* e, const int64_t* cell_lo,
                          int n_sub, const sub_variant* var, sub_ties* ties,
                          sub_work* wk, double res[4])
{
    int n_order = 0;
    double ta = tf->term_alpha;
    for (int i = 0; i < n_sub; ++i) {
        wk->C[3 * i] = wk->C[3 * i + 1] = wk->C[3 * i + 2] = 0.0;
        wk->A[i] = 0.0;
        wk->V[i] = mode == VRO_MIP ? -INFINITY : 0.0;
        wk->done[i] = 0;
    }
    int64_t* first_stop = NULL;  /* probe: the primary stop of each sub-cube */
    int64_t stops_buf[64];
    if (ties) {
        first_stop = n_sub <= 64 ? stops_buf : (int64_t*)malloc(sizeof(int64_t) * n_sub);
        for (int i = 0; i < n_sub; ++i) first_stop[i] = -1;
    }
    for (int64_t k = 0; k < K; ++k) {
        double t = t_entry + (double)k * step;
        double z = o[2] + t * d[2];
        int i = segment_of(z, cell_lo, n_sub);
        double sens[3];
        double s = sample_sens(vol, o, d, t, sens);
        if (ties) {
            double ep = pos_err(b, e, t, sens[2]) + ldexp(fabs(z) + 1.0, -22);
            for (int j = 1; j < n_sub; ++j) {
                double bz = (double)cell_lo[j];
                if (fabs(z - bz) <= ep) {
                    ties->flags |= 16;
                    if (ties->n_move < VRO_MAXMOVE) {
                        ties->move_k[ties->n_move] = k;
                        ties->move_to[ties->n_move++] = i >= j ? j - 1 : j;
                    } else {
                        ties->flags |= 8;
                    }
                }
            }
        }
        if (k == var->move_k) i = var->move_to;
        if (n_order == 0 || wk->order[n_order - 1] != i) wk->order[n_order++] = i;
        if (mode == VRO_MIP) {
            if (s > wk->V[i]) wk->V[i] = s;
            continue;
        }
        if (mode == VRO_SUM) {
            wk->V[i] += s * step;
            continue;
        }
        if (wk->done[i]) continue;
        int keep = !(s < tf->clip);
        if (ties && clip_alpha > 0.0 && clip_tie(b, e, tf, s, t, sens)) {
            ties->flags |= 2;
            if (ties->n_clip < VRO_MAXCLIP)
                ties->clip_k[ties->n_clip++] = k;
            else
                ties->flags |= 8;
        }
        if (k == var->flip_k) keep = !keep;
        if (!keep) continue;
        double rgba[4];
        classify(tf, lutc, s, rgba);
        double wgt = (1.0 - wk->A[i]) * rgba[3];
        for (int c = 0; c < 3; ++c) wk->C[3 * i + c] += wgt * rgba[c];
        wk->A[i] += wgt;
        double A = wk->A[i];
        if (ties) {
            if (A >= ta - b->band_a) {
                if (first_stop[i] < 0 && A >= ta) {
                    first_stop[i] = k;            /* the primary stop */
                } else {
                    ties->flags |= 4;
                    if (ties->n_stop < VRO_MAXSTOP) {
                        ties->stop_seg[ties->n_stop] = i;
                        ties->stop_k[ties->n_stop++] = k;
                    } else {
                        ties->flags |= 8;
                    }
                }
                if (A >= ta + b->band_a) wk->done[i] = 1;
            }
        } else if (i == var->stop_seg) {
            if (k == var->stop_k) wk->done[i] = 1;
        } else if (A >= ta) {
            wk->done[i] = 1;
        }
    }
    if (ties && first_stop != stops_buf) free(first_stop);
    /* combine each partial once, in the order of the ray's first visits (a
     * moved sample can make a ray revisit a sub-cube) */
    res[0] = res[1] = res[2] = res[3] = 0.0;
    if (mode == VRO_MIP) res[0] = -INFINITY;
    for (int a = 0; a < n_order; ++a) {
        int i = wk->order[a], seen = 0;
        for (int a2 = 0; a2 < a; ++a2) seen |= wk->order[a2] == i;
        if (seen) continue;
        if (mode == VRO_MIP) {
            if (wk->V[i] > res[0]) res[0] = wk->V[i];
        } else if (mode == VRO_SUM) {
            res[0] += wk->V[i];
        } else {
            double T = 1.0 - res[3];
            for (int c = 0; c < 3; ++c) res[c] += T * wk->C[3 * i + c];
            res[3] += T * wk->A[i];
        }
    }
}

static void render_pixel_subcubes(const vro_volume* vol, const vro_camera* cam, int w, int h,
                                  int px, int py, int mode, double step, const vro_tf* tf,
                                  const double* lutc, const vro_bands* b,
                                  const int64_t* cell_lo, int n_sub, alts* r, sub_work* wk)
{
    double o[3], d[3];
    make_ray(cam, w, h, px, py, o, d);
    double tn, tf_, miss_dist, face_dist, dn, df;
    slab(o, d, vol->n, &tn, &tf_, &miss_dist, &face_dist, &dn, &df);
    double t_entry = tn > 0.0 ? tn : 0.0;
    double q = (tf_ - t_entry) / step;
    int hit = miss_dist == 0.0 && tf_ >= t_entry;
    ray_err e = make_ray_err(b, o, tn, dn);
    double wq = b->band_k + (e.e_te + t_err(b, tf_, df)) / step;
    int64_t Ks[4];
    int nK = 0;
    if (hit) {
        double fl = floor(q);
        Ks[nK++] = (int64_t)fl + 1;
        if (q - fl < wq) Ks[nK++] = (int64_t)fl;
        if (q - fl > 1.0 - wq) Ks[nK++] = (int64_t)fl + 2;
        if (face_dist <= b->band_pos) Ks[nK++] = 0;
    } else {
        Ks[nK++] = 0;
        if (miss_dist <= b->band_pos && q >= -wq)
            Ks[nK++] = q < 0.0 ? 1 : (int64_t)floor(q) + 1;
    }
    r->n = 0;
    r->flags = nK > 1 ? 1 : 0;
    double clip_rgba[4];
    classify(tf, lutc, tf->clip, clip_rgba);
    sub_variant none = {-1, -1, 0, -1, -1};
    double res[4];
    subcube_march(vol, o, d, t_entry, Ks[0], step, mode, tf, lutc, clip_rgba[3], b, &e,
                  cell_lo, n_sub, &none, NULL, wk, res);
    push(r, res);
    for (int ik = 1; ik < nK; ++ik) {
        subcube_march(vol, o, d, t_entry, Ks[ik], step, mode, tf, lutc, clip_rgba[3], b, &e,
                      cell_lo, n_sub, &none, NULL, wk, res);
        push(r, res);
    }
    sub_ties ties;
    memset(&ties, 0, sizeof ties);
    subcube_march(vol, o, d, t_entry, Ks[0], step, mode, tf, lutc, clip_rgba[3], b, &e,
                  cell_lo, n_sub, &none, &ties, wk, res);
    r->flags |= ties.flags;
    for (int i = 0; i < ties.n_clip; ++i) {
        sub_variant v = none;
        v.flip_k = ties.clip_k[i];
        subcube_march(vol, o, d, t_entry, Ks[0], step, mode, tf, lutc, clip_rgba[3], b, &e,
                      cell_lo, n_sub, &v, NULL, wk, res);
        push(r, res);
    }
    for (int i = 0; i < ties.n_move; ++i) {
        sub_variant v = none;
        v.move_k = ties.move_k[i];
        v.move_to = ties.move_to[i];
        subcube_march(vol, o, d, t_entry, Ks[0], step, mode, tf, lutc, clip_rgba[3], b, &e,
                      cell_lo, n_sub, &v, NULL, wk, res);
        push(r, res);
    }
    for (int i = 0; i < ties.n_stop; ++i) {
        sub_variant v = none;
        v.stop_seg = ties.stop_seg[i];
        v.stop_k = ties.stop_k[i];
        subcube_march(vol, o, d, t_entry, Ks[0], step, mode, tf, lutc, clip_rgba[3], b, &e,
                      cell_lo, n_sub, &v, NULL, wk, res);
        push(r, res);
    }
}

/*
 * Render a list of pixels (as vro_render) as n_sub sub-cubes rendered
 * independently and integrated; cell_lo[0] must be 0 and cell_lo ascending
 * below n_z - 1.  Output as vro_render's: out[i*VRO_MAXALT*4 + a*4 + c] is
 * channel c of acceptable result a (a < nalt[i]; a = 0 the primary result;
 * MIP and SUM use channel 0).  Returns 0, or -1 on bad arguments.
 */
int vro_render_subcubes(const vro_volume* vol, const vro_camera* cams, int n_views, int w,
                        int h, int mode, double step, const vro_tf* tf,
                        const vro_bands* bands, const int64_t* cell_lo, int n_sub,
                        const int32_t* pix, int64_t npix, double* out, int32_t* nalt,
                        int32_t* flags, int nthreads)
{
    if (!vol || !cams || !tf || !bands || !cell_lo || !pix || !out || !nalt || !flags)
        return -1;
    if (vol->n[0] < 2 || vol->n[1] < 2 || vol->n[2] < 2 || !(step > 0.0) ||
        tf->n_lut < 2 || w <= 0 || h <= 0 || n_views <= 0 || n_sub < 1)
        return -1;
    if (mode != VRO_MIP && mode != VRO_COMPOSITE && mode != VRO_SUM) return -1;
    if (cell_lo[0] != 0) return -1;
    for (int i = 1; i < n_sub; ++i)
        if (!(cell_lo[i] > cell_lo[i - 1]) || cell_lo[i] >= vol->n[2] - 1) return -1;
    double* lutc = (double*)malloc(sizeof(double) * 4 * (size_t)tf->n_lut);
    if (!lutc) return -1;
    correct_table(tf, step, lutc);
    int bad = 0;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel num_threads(nt) reduction(| : bad)
#endif
    {
        sub_work wk;
        wk.C = (double*)malloc(sizeof(double) * 3 * (size_t)n_sub);
        wk.A = (double*)malloc(sizeof(double) * (size_t)n_sub);
        wk.V = (double*)malloc(sizeof(double) * (size_t)n_sub);
        wk.done = (int*)malloc(sizeof(int) * (size_t)n_sub);
        /* a ray visits each sub-cube in one run, but a moved sample can add
         * a visit: room for twice the sub-cubes */
        wk.order = (int*)malloc(sizeof(int) * 2 * (size_t)n_sub + 2 * sizeof(int));
        if (!wk.C || !wk.A || !wk.V || !wk.done || !wk.order) bad = 1;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t i = 0; i < npix; ++i) {
            int view = pix[3 * i], px = pix[3 * i + 1], py = pix[3 * i + 2];
            if (bad || view < 0 || view >= n_views || px < 0 || px >= w || py < 0 || py >= h) {
                bad = 1;
                continue;
            }
            alts r;
            render_pixel_subcubes(vol, &cams[view], w, h, px, py, mode, step, tf, lutc,
                                  bands, cell_lo, n_sub, &r, &wk);
            memset(&out[i * VRO_MAXALT * 4], 0, sizeof(double) * VRO_MAXALT * 4);
            for (int a = 0; a < r.n; ++a)
                memcpy(&out[(i * VRO_MAXALT + a) * 4], r.v[a], 4 * sizeof(double));
            nalt[i] = r.n;
            flags[i] = r.flags;
        }
        free(wk.C);
        free(wk.A);
        free(wk.V);
        free(wk.done);
        free(wk.order);
    }
    (void)nthreads;
    free(lutc);
    return bad ? -1 : 0;
}

/*
 * One sub-cube's partial result alone (the image a node of the paper's
 * pipeline renders for its sub-cube before scene integration, §3.1 item 4):
 * the primary FP64 result of sub-cube `part` of the split cell_lo[0..n_sub)
 * (as vro_render_subcubes), from an empty start, stopping at its own
 * opacity.  out[i*4 + c]: composite (C, A), MIP the maximum (-inf when no
 * sample falls in the sub-cube), SUM the sum, in channel 0.
 */
int vro_render_partial(const vro_volume* vol, const vro_camera* cams, int n_views, int w,
                       int h, int mode, double step, const vro_tf* tf, const int64_t* cell_lo,
                       int n_sub, int part, const int32_t* pix, int64_t npix, double* out,
                       int nthreads)
{
    if (!vol || !cams || !tf || !cell_lo || !pix || !out) return -1;
    if (vol->n[0] < 2 || vol->n[1] < 2 || vol->n[2] < 2 || !(step > 0.0) ||
        tf->n_lut < 2 || w <= 0 || h <= 0 || n_views <= 0 || n_sub < 1 || part < 0 ||
        part >= n_sub)
        return -1;
    if (mode != VRO_MIP && mode != VRO_COMPOSITE && mode != VRO_SUM) return -1;
    if (cell_lo[0] != 0) return -1;
    for (int i = 1; i < n_sub; ++i)
        if (!(cell_lo[i] > cell_lo[i - 1]) || cell_lo[i] >= vol->n[2] - 1) return -1;
    double* lutc = (double*)malloc(sizeof(double) * 4 * (size_t)tf->n_lut);
    if (!lutc) return -1;
    correct_table(tf, step, lutc);
    double clip_rgba[4];
    classify(tf, lutc, tf->clip, clip_rgba);
    const vro_bands none_b = {0.0, 0.0, 0.0, 0.0, 0.0};
    int bad = 0;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel num_threads(nt) reduction(| : bad)
#endif
    {
        sub_work wk;
        wk.C = (double*)malloc(sizeof(double) * 3 * (size_t)n_sub);
        wk.A = (double*)malloc(sizeof(double) * (size_t)n_sub);
        wk.V = (double*)malloc(sizeof(double) * (size_t)n_sub);
        wk.done = (int*)malloc(sizeof(int) * (size_t)n_sub);
        wk.order = (int*)malloc(sizeof(int) * 2 * (size_t)n_sub + 2 * sizeof(int));
        if (!wk.C || !wk.A || !wk.V || !wk.done || !wk.order) bad = 1;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t i = 0; i < npix; ++i) {
            int view = pix[3 * i], px = pix[3 * i + 1], py = pix[3 * i + 2];
            if (bad || view < 0 || view >= n_views || px < 0 || px >= w || py < 0 || py >= h) {
                bad = 1;
                continue;
            }
            double o[3], d[3];
            make_ray(&cams[view], w, h, px, py, o, d);
            double tn, tf_, miss_dist, face_dist, dn, df;
            slab(o, d, vol->n, &tn, &tf_, &miss_dist, &face_dist, &dn, &df);
            double t_entry = tn > 0.0 ? tn : 0.0;
            int64_t K = (miss_dist == 0.0 && tf_ >= t_entry)
                            ? (int64_t)floor((tf_ - t_entry) / step) + 1 : 0;
            ray_err e = make_ray_err(&none_b, o, tn, dn);
            sub_variant nv = {-1, -1, 0, -1, -1};
            double res[4];
            subcube_march(vol, o, d, t_entry, K, step, mode, tf, lutc, clip_rgba[3], &none_b,
                          &e, cell_lo, n_sub, &nv, NULL, &wk, res);
            double* r = &out[4 * i];
            if (mode == VRO_COMPOSITE) {
                r[0] = wk.C[3 * part];
                r[1] = wk.C[3 * part + 1];
                r[2] = wk.C[3 * part + 2];
                r[3] = wk.A[part];
            } else {
                r[0] = wk.V[part];
                r[1] = r[2] = r[3] = 0.0;
            }
        }
        free(wk.C);
        free(wk.A);
        free(wk.V);
        free(wk.done);
        free(wk.order);
    }
    (void)nthreads;
    free(lutc);
    return bad ? -1 : 0;
}

/* Exposed pieces for the oracle's own tests: one trilinear sample at a point
 * and the corrected table entry for a value.                             */
double vro_sample_at(const vro_volume* vol, double x, double y, double z)
{
    double o[3] = {x, y, z}, d[3] = {0, 0, 0};
    return sample(vol, o, d, 0.0);
}

void vro_classify(const vro_tf* tf, double step, double s, double* rgba)
{
    double* lutc = (double*)malloc(sizeof(double) * 4 * (size_t)tf->n_lut);
    if (!lutc) return;
    correct_table(tf, step, lutc);
    classify(tf, lutc, s, rgba);
    free(lutc);
}

double vro_half_to_double(uint16_t h) { return half_to_double(h); }

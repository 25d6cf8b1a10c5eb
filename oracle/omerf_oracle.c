/*
 * omerf_oracle.c -- plain, slow FP64 CPU oracle for the Oblique-MERF hot path
 * (Oblique-MERF: Revisiting and Improving MERF for Oblique Photography,
 * arXiv 2404.09531).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library; the product path never
 * calls it.  It shares no source, header, table or helper with the CUDA
 * library and includes nothing from it.
 *
 * What it evaluates, literally and in double precision:
 *   feature field   t(p) = V(p) + P_xy(p) + P_xz(p) + P_yz(p)        Sec. 3, Eq. 2
 *                   (trilinear grid, bilinear planes, vertex-aligned)
 *   activations     tau = exp(t0), c^d = sigmoid(t1..3), f = sigmoid(t4..7)   Eq. 3
 *   opacity         alpha = 1 - exp(-tau * delta)                     Sec. 3 (below Eq. 1)
 *   occupancy       M(z) power ramps with q = 2, nearest cell         Sec. 4.1, Eqs. 6-7
 *   compositing     w_i = T_i * M_i * alpha_i, T_{i+1} = T_i (1 - M_i alpha_i)   Eqs. 1, 8
 *   deferred MLP    C = sum w c^d + G(F, d), F = [sum w c^d, sum w f]  Eq. 4
 *   view encoding   [d, sin(2^k d), cos(2^k d)], k = 0..3             appendix A
 *   losses          Charbonnier (Eq. 12), view smoothness (Eqs. 9-10), L_occ (Eq. 5)
 *   gradient        reverse mode by hand (textbook back-to-front sweep)
 *   brick table     feature bricks stored where the occupancy plane says
 *                   "occupied" (Sec. 4.4)
 *   sparsity loss   mean opacity of given points in the occupied space (Eq. 13)
 *   entropy loss    -sum p log p along top-down rays, p = M alpha / sum M alpha (Eq. 14)
 *   extraction      3D occupancy grid from the occupancy plane (Sec. 5.3),
 *                   brick pool from a grid or an older pool, XZ/YZ plane rows
 *                   cropped to the occupancy bounds (Sec. 4.4)
 *
 * Readings of the paper taken here (all also used by the CUDA path):
 *   - the sample lattice is t_k = k * step (k >= 0) from the ray origin; which
 *     samples are evaluated is decided in FP32 arithmetic without fused
 *     multiply-add: p_k = o + t_k d, AABB test (closed), nearest occupancy
 *     cell = floor((x - x0) * (M / (x1 - x0))), test z_min < z < z_max
 *     (strict).  Everything after that decision is FP64.
 *   - M enters through alpha: alpha_hat = M * alpha, and the transmittance is
 *     built from alpha_hat (so sum w + T_N = 1).
 *   - where the two ramps of Eq. 6 overlap (z_max - z_min < 2 eps) the value
 *     is min(1, r_lo^2, r_hi^2); elsewhere this is Eq. 6 exactly.
 *   - a ray stops after the sample at which T drops below t_thr (t_thr = 0
 *     disables this), or after n_max evaluated samples.
 *   - a ray with no evaluated sample returns the background and skips G.
 *   - the output is C = sum w c^d + G(F, d) + T_N * bg.
 *   - losses are means over the rays of a batch (L_occ is a sum over cells).
 *
 * Build: cc -O2 -std=c11 -fPIC -shared -ffp-contract=off -fopenmp
 * (-ffp-contract=off is required: the FP32 sample decisions must not fuse).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NCH 8
#define NIN 34
#define NHID 16
#define NOUT 3
#define NPARAM 883
/* MLP parameter offsets: W1[16][34] b1[16] W2[16][16] b2[16] W3[3][16] b3[3] */
#define OFF_W1 0
#define OFF_B1 544
#define OFF_W2 560
#define OFF_B2 816
#define OFF_W3 832
#define OFF_B3 880
#define AMBIG_BAND 1e-4
#define CHARB_EPS 1e-6

typedef struct {
    float aabb[6];           /* x0 x1 y0 y1 z0 z1 */
    int32_t L[3];            /* grid vertices per axis (>= 2) */
    int32_t brick;           /* brick edge in vertices; 0 = dense grid */
    const int32_t *table;    /* brick -> pool index or -1 (brick grids only) */
    const double *grid;      /* dense [Lx][Ly][Lz][8] or pool [nb][B][B][B][8] */
    int32_t R[3];            /* plane texels: XY Rx x Ry, XZ Rx x Rz, YZ Ry x Rz */
    const double *pxy, *pxz, *pyz;
    int32_t M;               /* occupancy cells per axis */
    const double *occ;       /* [M][M][2]: z_min, z_max */
    const double *mlp;       /* 883 parameters */
    float step;              /* lattice spacing, a power of two */
    float eps;               /* occupancy ramp width */
    float t_thr;             /* early termination threshold on T; 0 = off */
    float bg[3];             /* background colour */
    int32_t n_max;           /* maximum evaluated samples per ray */
    float pz[2];             /* z-range spanned by the XZ and YZ planes; pz[1] <= pz[0]: the box's */
} or_scene;

/* one evaluated sample, kept for the backward sweep */
typedef struct {
    double p[3];
    int cell;                /* occupancy cell index ix * M + iy */
    int branch;              /* 0: M = 1, 1: lower ramp, 2: upper ramp */
    double r;                /* ramp coordinate of the active branch */
    double Mv, tau, sigma, alpha, ah, T;
    double x[7];             /* c^d (3), f (4) */
} or_sample;

typedef struct {
    int count;
    int ambiguous;
    int k_first, k_last;     /* lattice indices of first / last evaluated sample */
    double F[7];
    double TN;
    long unalloc;            /* corner reads of unallocated bricks */
} or_march;

static const double ZERO8[NCH] = {0, 0, 0, 0, 0, 0, 0, 0};

/* ------------------------------------------------------------------ */
/* feature field (Eq. 2)                                               */
/* ------------------------------------------------------------------ */

/* vertex-aligned coordinate along one axis: u = (x - lo)/(hi - lo) * (L - 1),
 * clamped to [0, L-1]; corners i0 and i0 + 1 with i0 <= L - 2. */
static void axis_coord(double x, double lo, double hi, int L, int *i0, double *w)
{
    double u = (x - lo) / (hi - lo) * (double)(L - 1);
    if (u < 0.0) u = 0.0;
    if (u > (double)(L - 1)) u = (double)(L - 1);
    int i = (int)floor(u);
    if (i > L - 2) i = L - 2;
    *i0 = i;
    *w = u - (double)i;
}

static long grid_vertex_index(const or_scene *s, int i, int j, int k, int *unalloc)
{
    if (s->brick == 0)
        return (((long)i * s->L[1] + j) * s->L[2] + k) * NCH;
    int B = s->brick;
    int nbj = (s->L[1] + B - 1) / B, nbk = (s->L[2] + B - 1) / B;
    int b = s->table[((long)(i / B) * nbj + j / B) * nbk + k / B];
    if (b < 0) {
        if (unalloc) (*unalloc)++;
        return -1;
    }
    return ((((long)b * B + i % B) * B + j % B) * B + k % B) * NCH;
}

typedef struct {
    /* grid corners */
    long gidx[8];
    double gw[8];
    /* plane texels: XY, XZ, YZ, 4 each */
    long pidx[3][4];
    double pw[3][4];
} or_stencil;

static void make_stencil(const or_scene *s, const double p[3], or_stencil *st, int *unalloc)
{
    const float *a = s->aabb;
    int gi[3];
    double gw[3];
    for (int d = 0; d < 3; d++)
        axis_coord(p[d], a[2 * d], a[2 * d + 1], s->L[d], &gi[d], &gw[d]);
    int n = 0;
    for (int da = 0; da < 2; da++)
        for (int db = 0; db < 2; db++)
            for (int dc = 0; dc < 2; dc++) {
                double w = (da ? gw[0] : 1.0 - gw[0]) * (db ? gw[1] : 1.0 - gw[1]) *
                           (dc ? gw[2] : 1.0 - gw[2]);
                st->gidx[n] = grid_vertex_index(s, gi[0] + da, gi[1] + db, gi[2] + dc, unalloc);
                st->gw[n] = w;
                n++;
            }
    int pi[3];
    double pw[3];
    for (int d = 0; d < 2; d++)
        axis_coord(p[d], a[2 * d], a[2 * d + 1], s->R[d], &pi[d], &pw[d]);
    if (s->pz[1] > s->pz[0])
        axis_coord(p[2], s->pz[0], s->pz[1], s->R[2], &pi[2], &pw[2]);
    else
        axis_coord(p[2], a[4], a[5], s->R[2], &pi[2], &pw[2]);
    /* plane q spans axes (ax0, ax1): XY (0,1), XZ (0,2), YZ (1,2) */
    static const int AX[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int q = 0; q < 3; q++) {
        int u = AX[q][0], v = AX[q][1];
        int m = 0;
        for (int da = 0; da < 2; da++)
            for (int db = 0; db < 2; db++) {
                st->pidx[q][m] = ((long)(pi[u] + da) * s->R[v] + (pi[v] + db)) * NCH;
                st->pw[q][m] = (da ? pw[u] : 1.0 - pw[u]) * (db ? pw[v] : 1.0 - pw[v]);
                m++;
            }
    }
}

static const double *plane_ptr(const or_scene *s, int q)
{
    return q == 0 ? s->pxy : (q == 1 ? s->pxz : s->pyz);
}

static void eval_features(const or_scene *s, const or_stencil *st, double t[NCH])
{
    for (int c = 0; c < NCH; c++) t[c] = 0.0;
    for (int n = 0; n < 8; n++) {
        const double *v = st->gidx[n] < 0 ? ZERO8 : s->grid + st->gidx[n];
        for (int c = 0; c < NCH; c++) t[c] += st->gw[n] * v[c];
    }
    for (int q = 0; q < 3; q++) {
        const double *P = plane_ptr(s, q);
        for (int m = 0; m < 4; m++)
            for (int c = 0; c < NCH; c++) t[c] += st->pw[q][m] * P[st->pidx[q][m] + c];
    }
}

/* ------------------------------------------------------------------ */
/* occupancy function (Eq. 6, q = 2)                                   */
/* ------------------------------------------------------------------ */
static double occupancy_value(double z, double zmin, double zmax, double eps, int *branch, double *r)
{
    if (!(z > zmin && z < zmax)) {
        *branch = -1;
        *r = 0.0;
        return 0.0;
    }
    double rl = (z - zmin) / eps, rh = (zmax - z) / eps;
    double ml = rl * rl, mh = rh * rh;
    if (ml < 1.0 && ml <= mh) {
        *branch = 1;
        *r = rl;
        return ml;
    }
    if (mh < 1.0) {
        *branch = 2;
        *r = rh;
        return mh;
    }
    *branch = 0;
    *r = 0.0;
    return 1.0;
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* ------------------------------------------------------------------ */
/* FP32 sample schedule (the decisions; no fused multiply-add)         */
/* ------------------------------------------------------------------ */

/* slab method in FP64, used only to bound the brute-force lattice scan */
static int slab_range(const or_scene *s, const float o[3], const float d[3], double *tin, double *tout)
{
    double t0 = -INFINITY, t1 = INFINITY;
    for (int a = 0; a < 3; a++) {
        double lo = s->aabb[2 * a], hi = s->aabb[2 * a + 1];
        if (d[a] == 0.0f) {
            if (o[a] < lo || o[a] > hi) return 0;
            continue;
        }
        double ta = (lo - o[a]) / d[a], tb = (hi - o[a]) / d[a];
        if (ta > tb) { double x = ta; ta = tb; tb = x; }
        /* widen by far more than the FP32 error of the sample positions, so
         * that the scan covers every lattice point the FP32 test accepts */
        double pad = 1e-6 * (fmax(fabs(ta), fabs(tb)) + (fabs((double)o[a]) + 1.0) / fabs((double)d[a]));
        ta -= pad;
        tb += pad;
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
    }
    if (t1 < 0.0 || t0 > t1) return 0;
    *tin = t0;
    *tout = t1;
    return 1;
}

/* is lattice sample k evaluated by occupancy/box rules? writes p and cell */
static int lattice_test(const or_scene *s, const float o[3], const float d[3], long k,
                        float p[3], int *cell)
{
    float t = (float)k * s->step;  /* exact: step is a power of two, k < 2^24 */
    for (int a = 0; a < 3; a++) p[a] = o[a] + t * d[a];
    const float *b = s->aabb;
    if (!(p[0] >= b[0] && p[0] <= b[1] && p[1] >= b[2] && p[1] <= b[3] && p[2] >= b[4] && p[2] <= b[5]))
        return 0;
    float sx = (float)s->M / (b[1] - b[0]);
    float sy = (float)s->M / (b[3] - b[2]);
    int cx = (int)floorf((p[0] - b[0]) * sx);
    int cy = (int)floorf((p[1] - b[2]) * sy);
    if (cx < 0) cx = 0;
    if (cx > s->M - 1) cx = s->M - 1;
    if (cy < 0) cy = 0;
    if (cy > s->M - 1) cy = s->M - 1;
    *cell = cx * s->M + cy;
    float zmin = (float)s->occ[2 * (*cell)], zmax = (float)s->occ[2 * (*cell) + 1];
    return zmin < p[2] && p[2] < zmax;
}

/* march one ray: every lattice index from a margin before box entry to a
 * margin after box exit is tested; no skipping. */
static void march_ray(const or_scene *s, const float ray[6], or_sample *smp, or_march *out)
{
    memset(out, 0, sizeof(*out));
    out->k_first = out->k_last = -1;
    out->TN = 1.0;
    const float *o = ray, *d = ray + 3;
    double tin, tout;
    if (!slab_range(s, o, d, &tin, &tout)) return;
    /* lattice indices are limited to k < 2^24, where k * step is exact */
    double fklo = floor(tin / s->step) - 2.0, fkhi = ceil(tout / s->step) + 2.0;
    if (fklo < 0.0) fklo = 0.0;
    if (fkhi > 16777215.0) fkhi = 16777215.0;
    if (fklo > fkhi) return;
    long klo = (long)fklo, khi = (long)fkhi;
    double T = 1.0;
    int n = 0;
    for (long k = klo; k <= khi; k++) {
        float p32[3];
        int cell;
        if (!lattice_test(s, o, d, k, p32, &cell)) continue;
        if (n >= s->n_max) break;
        or_sample *q = &smp[n];
        for (int a = 0; a < 3; a++) q->p[a] = (double)p32[a];
        q->cell = cell;
        q->Mv = occupancy_value(q->p[2], s->occ[2 * cell], s->occ[2 * cell + 1], (double)s->eps,
                                &q->branch, &q->r);
        or_stencil st;
        int ua = 0;
        make_stencil(s, q->p, &st, &ua);
        out->unalloc += ua;
        double t[NCH];
        eval_features(s, &st, t);
        q->tau = exp(t[0]);
        q->sigma = q->tau * (double)s->step;
        q->alpha = -expm1(-q->sigma);
        q->ah = q->Mv * q->alpha;
        for (int c = 0; c < 7; c++) q->x[c] = sigmoid(t[c + 1]);
        q->T = T;
        double w = T * q->ah;
        for (int c = 0; c < 7; c++) out->F[c] += w * q->x[c];
        T *= 1.0 - q->ah;
        if (out->k_first < 0) out->k_first = (int)k;
        out->k_last = (int)k;
        n++;
        if (s->t_thr > 0.0f) {
            if (fabs(T / (double)s->t_thr - 1.0) < AMBIG_BAND) out->ambiguous = 1;
            if (T < (double)s->t_thr) break;
        }
    }
    out->count = n;
    out->TN = T;
}

/* ------------------------------------------------------------------ */
/* deferred MLP G (Eq. 4; 3 layers of 16 units, appendix A)            */
/* ------------------------------------------------------------------ */
static void view_encoding(const double d[3], double enc[27])
{
    for (int a = 0; a < 3; a++) enc[a] = d[a];
    for (int k = 0; k < 4; k++) {
        double f = ldexp(1.0, k);
        for (int a = 0; a < 3; a++) {
            enc[3 + 6 * k + a] = sin(f * d[a]);
            enc[3 + 6 * k + 3 + a] = cos(f * d[a]);
        }
    }
}

typedef struct {
    double x[NIN], a1[NHID], h1[NHID], a2[NHID], h2[NHID], a3[NOUT], y[NOUT];
} or_mlp_cache;

static void mlp_forward(const double *P, const double F[7], const double dir[3], or_mlp_cache *c)
{
    for (int i = 0; i < 7; i++) c->x[i] = F[i];
    view_encoding(dir, c->x + 7);
    for (int j = 0; j < NHID; j++) {
        double a = P[OFF_B1 + j];
        for (int i = 0; i < NIN; i++) a += P[OFF_W1 + j * NIN + i] * c->x[i];
        c->a1[j] = a;
        c->h1[j] = a > 0.0 ? a : 0.0;
    }
    for (int j = 0; j < NHID; j++) {
        double a = P[OFF_B2 + j];
        for (int i = 0; i < NHID; i++) a += P[OFF_W2 + j * NHID + i] * c->h1[i];
        c->a2[j] = a;
        c->h2[j] = a > 0.0 ? a : 0.0;
    }
    for (int j = 0; j < NOUT; j++) {
        double a = P[OFF_B3 + j];
        for (int i = 0; i < NHID; i++) a += P[OFF_W3 + j * NHID + i] * c->h2[i];
        c->a3[j] = a;
        c->y[j] = sigmoid(a);
    }
}

/* textbook backprop of gy through the cached forward; adds into gP (may be
 * NULL) and returns the gradient w.r.t. the 7 feature inputs in gF */
static void mlp_backward(const double *P, const or_mlp_cache *c, const double gy[NOUT], double *gP,
                         double gF[7])
{
    double g3[NOUT], gh2[NHID], g2[NHID], gh1[NHID], g1[NHID];
    for (int j = 0; j < NOUT; j++) g3[j] = gy[j] * c->y[j] * (1.0 - c->y[j]);
    for (int i = 0; i < NHID; i++) {
        double a = 0.0;
        for (int j = 0; j < NOUT; j++) a += P[OFF_W3 + j * NHID + i] * g3[j];
        gh2[i] = a;
        g2[i] = c->a2[i] > 0.0 ? a : 0.0;
    }
    for (int i = 0; i < NHID; i++) {
        double a = 0.0;
        for (int j = 0; j < NHID; j++) a += P[OFF_W2 + j * NHID + i] * g2[j];
        gh1[i] = a;
        g1[i] = c->a1[i] > 0.0 ? a : 0.0;
    }
    for (int i = 0; i < 7; i++) {
        double a = 0.0;
        for (int j = 0; j < NHID; j++) a += P[OFF_W1 + j * NIN + i] * g1[j];
        gF[i] += a;
    }
    if (!gP) return;
    for (int j = 0; j < NOUT; j++) {
        gP[OFF_B3 + j] += g3[j];
        for (int i = 0; i < NHID; i++) gP[OFF_W3 + j * NHID + i] += g3[j] * c->h2[i];
    }
    for (int j = 0; j < NHID; j++) {
        gP[OFF_B2 + j] += g2[j];
        for (int i = 0; i < NHID; i++) gP[OFF_W2 + j * NHID + i] += g2[j] * c->h1[i];
    }
    for (int j = 0; j < NHID; j++) {
        gP[OFF_B1 + j] += g1[j];
        for (int i = 0; i < NIN; i++) gP[OFF_W1 + j * NIN + i] += g1[j] * c->x[i];
    }
}

static uint64_t sig_mix(uint64_t h, uint64_t v)
{
    h ^= v + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
    return h;
}

static uint64_t mlp_signature(uint64_t h, const or_mlp_cache *c)
{
    uint64_t bits = 0;
    for (int j = 0; j < NHID; j++) bits |= (uint64_t)(c->a1[j] > 0.0) << j;
    for (int j = 0; j < NHID; j++) bits |= (uint64_t)(c->a2[j] > 0.0) << (16 + j);
    return sig_mix(h, bits);
}

/* ------------------------------------------------------------------ */
/* public entry points                                                 */
/* ------------------------------------------------------------------ */

int or_mlp_param_count(void) { return NPARAM; }

/* Eq. 6 at one point (q = 2) */
double or_occupancy_value(double z, double zmin, double zmax, double eps)
{
    int b;
    double r;
    return occupancy_value(z, zmin, zmax, eps, &b, &r);
}

/* the view encoding of a direction (27 values) */
void or_view_encoding(const double *dir, double *enc) { view_encoding(dir, enc); }

/* G(F, d) for n inputs: F [n][7], dir [n][3] -> out [n][3] */
void or_mlp(const double *P, const double *F, const double *dir, long n, double *out)
{
    for (long r = 0; r < n; r++) {
        or_mlp_cache c;
        mlp_forward(P, F + 7 * r, dir + 3 * r, &c);
        for (int j = 0; j < 3; j++) out[3 * r + j] = c.y[j];
    }
}

/* the summed feature t(p) of Eq. 2 at n points [n][3] -> [n][8]; returns
 * the number of unallocated-brick corner reads */
long or_features(const or_scene *s, const double *pts, long n, double *out)
{
    long ua_total = 0;
    for (long r = 0; r < n; r++) {
        or_stencil st;
        int ua = 0;
        make_stencil(s, pts + 3 * r, &st, &ua);
        ua_total += ua;
        eval_features(s, &st, out + NCH * r);
    }
    return ua_total;
}

/* pinhole rays for a W x H image, pixel centres, row-major pixel order.
 * cam = c2w (3x4 row-major) then fx, fy, cx, cy.  FP32, no fused ops. */
void or_camera_rays(const float *cam, int W, int H, float *rays)
{
    for (int py = 0; py < H; py++)
        for (int px = 0; px < W; px++) {
            float ux = ((float)px + 0.5f - cam[14]) / cam[12];
            float uy = -(((float)py + 0.5f - cam[15]) / cam[13]);
            float uz = -1.0f;
            float dx = (cam[0] * ux + cam[1] * uy) + cam[2] * uz;
            float dy = (cam[4] * ux + cam[5] * uy) + cam[6] * uz;
            float dz = (cam[8] * ux + cam[9] * uy) + cam[10] * uz;
            float nn = sqrtf((dx * dx + dy * dy) + dz * dz);
            float *r = rays + 6 * ((long)py * W + px);
            r[0] = cam[3];
            r[1] = cam[7];
            r[2] = cam[11];
            r[3] = dx / nn;
            r[4] = dy / nn;
            r[5] = dz / nn;
        }
}

/* threads of a parallel region: nthreads > 0 asks for that many for this
 * call only, 0 for the OpenMP default */
static int team_size(int nthreads)
{
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* forward render of n rays [n][6].  Outputs (any may be NULL except rgb):
 * rgb [n][3], count [n], F [n][7], TN [n], ambiguous [n], k_first/k_last [n].
 * Returns the total number of unallocated-brick corner reads. */
long or_render(const or_scene *s, const float *rays, long n, double *rgb, int32_t *count, double *F,
               double *TN, int32_t *ambiguous, int32_t *k_first, int32_t *k_last, int nthreads)
{
    long ua_total = 0;
    const int nt = team_size(nthreads);
#pragma omp parallel num_threads(nt) reduction(+ : ua_total)
    {
        or_sample *smp = (or_sample *)malloc(sizeof(or_sample) * (size_t)(s->n_max > 0 ? s->n_max : 1));
#pragma omp for schedule(dynamic, 64)
        for (long r = 0; r < n; r++) {
            or_march m;
            march_ray(s, rays + 6 * r, smp, &m);
            ua_total += m.unalloc;
            double out[3];
            if (m.count == 0) {
                for (int j = 0; j < 3; j++) out[j] = s->bg[j];
            } else {
                double dir[3] = {rays[6 * r + 3], rays[6 * r + 4], rays[6 * r + 5]};
                or_mlp_cache c;
                mlp_forward(s->mlp, m.F, dir, &c);
                for (int j = 0; j < 3; j++) out[j] = m.F[j] + c.y[j] + m.TN * s->bg[j];
            }
            for (int j = 0; j < 3; j++) rgb[3 * r + j] = out[j];
            if (count) count[r] = m.count;
            if (F)
                for (int j = 0; j < 7; j++) F[7 * r + j] = m.F[j];
            if (TN) TN[r] = m.TN;
            if (ambiguous) ambiguous[r] = m.ambiguous;
            if (k_first) k_first[r] = m.k_first;
            if (k_last) k_last[r] = m.k_last;
        }
        free(smp);
    }
    return ua_total;
}

/* Compositing weights of one ray (for invariant checks): w [n_max], returns
 * count; TN receives the final transmittance. */
int or_ray_weights(const or_scene *s, const float *ray, double *w, double *TN)
{
    or_sample *smp = (or_sample *)malloc(sizeof(or_sample) * (size_t)(s->n_max > 0 ? s->n_max : 1));
    or_march m;
    march_ray(s, ray, smp, &m);
    for (int i = 0; i < m.count; i++) w[i] = smp[i].T * smp[i].ah;
    *TN = m.TN;
    free(smp);
    return m.count;
}

/*
 * Training loss and its gradient for n rays.
 *   L = lam[0] * mean_r sqrt(|C_r - C*_r|^2 + 1e-6)                      (Eq. 12)
 *     + lam[1] * mean_r sum_k S(d, s_k) |G(F, s_k/|s_k|) - G(F, d)|^2    (Eqs. 9-10)
 *     + lam[2] * sum_cells (z_max - z_min)^2                              (Eq. 5)
 * smooth: [n][K][3] perturbed directions s = d + delta (raw, not normalised).
 * loss_out[4] = total, rgb term, smoothness term, occupancy term (weighted).
 * Gradients (any may be NULL) ACCUMULATE grad_scale * dL/dparam.
 * sig (may be NULL) receives a hash of every discrete decision (counts,
 * ramp branches, ReLU patterns) for finite-difference screening.
 */
int or_train(const or_scene *s, const float *rays, const float *target, const float *smooth, long n, int K,
             const double *lam, double grad_scale, double *loss_out, double *g_grid, double *g_xy,
             double *g_xz, double *g_yz, double *g_occ, double *g_mlp, uint64_t *sig)
{
    or_sample *smp = (or_sample *)malloc(sizeof(or_sample) * (size_t)(s->n_max > 0 ? s->n_max : 1));
    or_mlp_cache *cs = (or_mlp_cache *)malloc(sizeof(or_mlp_cache) * (size_t)(K > 0 ? K : 1));
    if (!smp || !cs) return -1;
    double l_rgb = 0.0, l_smooth = 0.0, l_occ = 0.0;
    uint64_t h = 1469598103934665603ULL;
    const double inv_n = n > 0 ? 1.0 / (double)n : 0.0;
    int want_grad = g_grid || g_xy || g_xz || g_yz || g_occ || g_mlp;
    for (long r = 0; r < n; r++) {
        const float *ray = rays + 6 * r;
        or_march m;
        march_ray(s, ray, smp, &m);
        h = sig_mix(h, (uint64_t)m.count);
        for (int i = 0; i < m.count; i++) h = sig_mix(h, (uint64_t)(smp[i].branch + 7 * smp[i].cell));
        double C[3];
        const float *tg = target + 3 * r;
        if (m.count == 0) {
            double e2 = 0.0;
            for (int j = 0; j < 3; j++) {
                double e = (double)s->bg[j] - (double)tg[j];
                e2 += e * e;
            }
            l_rgb += sqrt(e2 + CHARB_EPS);
            continue;
        }
        double dir[3] = {ray[3], ray[4], ray[5]};
        or_mlp_cache cd;
        mlp_forward(s->mlp, m.F, dir, &cd);
        h = mlp_signature(h, &cd);
        for (int j = 0; j < 3; j++) C[j] = m.F[j] + cd.y[j] + m.TN * s->bg[j];
        double e[3], e2 = 0.0;
        for (int j = 0; j < 3; j++) {
            e[j] = C[j] - tg[j];
            e2 += e[j] * e[j];
        }
        double ell = sqrt(e2 + CHARB_EPS);
        l_rgb += ell;
        /* smoothness terms */
        double gyd[3] = {0, 0, 0};
        double gys[16][3];
        double dn = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
        for (int k = 0; k < K; k++) {
            const float *sv = smooth + 3 * ((long)r * K + k);
            double sr[3] = {sv[0], sv[1], sv[2]};
            double sn = sqrt(sr[0] * sr[0] + sr[1] * sr[1] + sr[2] * sr[2]);
            double shat[3] = {sr[0] / sn, sr[1] / sn, sr[2] / sn};
            double S = (dir[0] * sr[0] + dir[1] * sr[1] + dir[2] * sr[2]) / (dn * sn);
            mlp_forward(s->mlp, m.F, shat, &cs[k]);
            h = mlp_signature(h, &cs[k]);
            double diff2 = 0.0;
            for (int j = 0; j < 3; j++) {
                double df = cs[k].y[j] - cd.y[j];
                diff2 += df * df;
                if (k < 16) gys[k][j] = lam[1] * inv_n * grad_scale * 2.0 * S * df;
            }
            l_smooth += S * diff2;
        }
        if (!want_grad) continue;
        /* dL/dC */
        double gC[3];
        for (int j = 0; j < 3; j++) gC[j] = lam[0] * inv_n * grad_scale * e[j] / ell;
        double gF[7] = {gC[0], gC[1], gC[2], 0, 0, 0, 0};
        for (int j = 0; j < 3; j++) gyd[j] = gC[j];
        for (int k = 0; k < K && k < 16; k++)
            for (int j = 0; j < 3; j++) gyd[j] -= gys[k][j];
        mlp_backward(s->mlp, &cd, gyd, g_mlp, gF);
        for (int k = 0; k < K && k < 16; k++) mlp_backward(s->mlp, &cs[k], gys[k], g_mlp, gF);
        double gT = gC[0] * s->bg[0] + gC[1] * s->bg[1] + gC[2] * s->bg[2];
        /* back-to-front sweep: Q = d(L)/d(radiance arriving just behind sample i) */
        double Q = gT;
        for (int i = m.count - 1; i >= 0; i--) {
            const or_sample *q = &smp[i];
            double gx = 0.0;
            for (int c = 0; c < 7; c++) gx += gF[c] * q->x[c];
            double dah = q->T * (gx - Q);
            Q = q->ah * gx + (1.0 - q->ah) * Q;
            double w = q->T * q->ah;
            double dt[NCH];
            double dsig = dah * q->Mv * (1.0 - q->alpha);
            dt[0] = dsig * q->sigma;
            for (int c = 0; c < 7; c++) dt[c + 1] = w * gF[c] * q->x[c] * (1.0 - q->x[c]);
            double dM = dah * q->alpha;
            if (g_occ) {
                if (q->branch == 1) g_occ[2 * q->cell] += dM * (-2.0 * q->r / (double)s->eps);
                if (q->branch == 2) g_occ[2 * q->cell + 1] += dM * (2.0 * q->r / (double)s->eps);
            }
            or_stencil st;
            make_stencil(s, q->p, &st, NULL);
            if (g_grid)
                for (int a = 0; a < 8; a++) {
                    if (st.gidx[a] < 0) continue;
                    for (int c = 0; c < NCH; c++) g_grid[st.gidx[a] + c] += st.gw[a] * dt[c];
                }
            double *gp[3] = {g_xy, g_xz, g_yz};
            for (int pq = 0; pq < 3; pq++) {
                if (!gp[pq]) continue;
                for (int a = 0; a < 4; a++)
                    for (int c = 0; c < NCH; c++) gp[pq][st.pidx[pq][a] + c] += st.pw[pq][a] * dt[c];
            }
        }
    }
    long ncell = (long)s->M * s->M;
    for (long c = 0; c < ncell; c++) {
        double span = s->occ[2 * c + 1] - s->occ[2 * c];
        l_occ += span * span;
        if (g_occ) {
            g_occ[2 * c + 1] += grad_scale * lam[2] * 2.0 * span;
            g_occ[2 * c] -= grad_scale * lam[2] * 2.0 * span;
        }
    }
    double lr = lam[0] * l_rgb * inv_n, ls = lam[1] * l_smooth * inv_n, lo = lam[2] * l_occ;
    if (loss_out) {
        loss_out[0] = lr + ls + lo;
        loss_out[1] = lr;
        loss_out[2] = ls;
        loss_out[3] = lo;
    }
    if (sig) *sig = h;
    free(smp);
    free(cs);
    return 0;
}

/*
 * Occupancy-driven brick allocation (Sec. 4.4): brick (bi, bj, bk) of B^3
 * vertices is stored iff some occupancy cell overlapping the brick's xy
 * footprint dilated by one voxel has a non-empty [z_min, z_max] that meets
 * the brick's z-range dilated by one voxel.  The cell range follows from
 * exact integer arithmetic (cell i covers [i, i+1) * (x1-x0)/M); the z test
 * is FP32 without fused operations.  Pool indices are assigned in x-major
 * brick order.  Returns the number of allocated bricks.
 */
static long floor_div(long a, long b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

long or_brick_table(const float *aabb, const int32_t *L, int B, const float *occ, int M, int32_t *table)
{
    int nb[3];
    for (int a = 0; a < 3; a++) nb[a] = (L[a] + B - 1) / B;
    float vz = (aabb[5] - aabb[4]) / (float)(L[2] - 1);
    long next = 0;
    for (int bi = 0; bi < nb[0]; bi++)
        for (int bj = 0; bj < nb[1]; bj++)
            for (int bk = 0; bk < nb[2]; bk++) {
                long lo[2], hi[2];
                int bb[2] = {bi, bj};
                for (int a = 0; a < 2; a++) {
                    /* cell i overlaps [v0 - 1, v0 + B] (vertex units) iff
                     * i <= (v0 + B) * M / (L - 1) and i + 1 >= (v0 - 1) * M / (L - 1) */
                    long v0 = (long)bb[a] * B;
                    long den = L[a] - 1;
                    lo[a] = -floor_div(-((v0 - 1) * (long)M), den) - 1;
                    hi[a] = floor_div((v0 + B) * (long)M, den);
                    if (lo[a] < 0) lo[a] = 0;
                    if (hi[a] > M - 1) hi[a] = M - 1;
                }
                float zlo = aabb[4] + (float)(bk * B - 1) * vz;
                float zhi = aabb[4] + (float)(bk * B + B) * vz;
                int hit = 0;
                for (long i = lo[0]; i <= hi[0] && !hit; i++)
                    for (long j = lo[1]; j <= hi[1] && !hit; j++) {
                        float zmin = occ[2 * (i * M + j)], zmax = occ[2 * (i * M + j) + 1];
                        if (zmin <= zmax && zmax >= zlo && zmin <= zhi) hit = 1;
                    }
                table[((long)bi * nb[1] + bj) * nb[2] + bk] = hit ? (int32_t)next++ : -1;
            }
    return next;
}

/* ------------------------------------------------------------------ */
/* regularisers of Sec. 4.3                                            */
/* ------------------------------------------------------------------ */

static void scatter_stencil(const or_scene *s, const or_stencil *st, const double dt[NCH], double *g_grid,
                            double *g_xy, double *g_xz, double *g_yz)
{
    if (g_grid)
        for (int a = 0; a < 8; a++) {
            if (st->gidx[a] < 0) continue;
            for (int c = 0; c < NCH; c++) g_grid[st->gidx[a] + c] += st->gw[a] * dt[c];
        }
    double *gp[3] = {g_xy, g_xz, g_yz};
    for (int q = 0; q < 3; q++) {
        if (!gp[q]) continue;
        for (int a = 0; a < 4; a++)
            for (int c = 0; c < NCH; c++) gp[q][st->pidx[q][a] + c] += st->pw[q][a] * dt[c];
    }
}

/*
 * Sparsity loss (Eq. 13): L = lam / n * sum_i alpha(p_i), alpha = 1 -
 * exp(-tau(p) delta) with delta the lattice step (reading: the opacity a
 * sample at p would have).  Points [n][3] are given by the caller.
 * Returns L; gradients (may be NULL) accumulate grad_scale * dL/dparam.
 */
double or_sparsity(const or_scene *s, const double *pts, long n, double lam, double grad_scale, double *g_grid,
                   double *g_xy, double *g_xz, double *g_yz)
{
    double acc = 0.0;
    for (long i = 0; i < n; i++) {
        or_stencil st;
        make_stencil(s, pts + 3 * i, &st, NULL);
        double t[NCH];
        eval_features(s, &st, t);
        double sigma = exp(t[0]) * (double)s->step;
        double alpha = -expm1(-sigma);
        acc += alpha;
        double dt[NCH] = {0, 0, 0, 0, 0, 0, 0, 0};
        dt[0] = grad_scale * lam / (double)n * (1.0 - alpha) * sigma;
        scatter_stencil(s, &st, dt, g_grid, g_xy, g_xz, g_yz);
    }
    return n > 0 ? lam * acc / (double)n : 0.0;
}

/*
 * Entropy loss (Eq. 14) over n rays: for each ray, a_i = M_i alpha_i over its
 * evaluated samples (no early termination; the n_max cap applies), p_i =
 * a_i / S with S = sum a_i, L_r = -sum p_i log p_i; L = lam / n * sum_r L_r.
 * Rays with S = 0 contribute 0.  dL_r/da_k = -(log p_k + L_r) / S.
 * Returns L; gradients (may be NULL) accumulate grad_scale * dL/dparam.
 */
double or_entropy(const or_scene *s, const float *rays, long n, double lam, double grad_scale, double *g_grid,
                  double *g_xy, double *g_xz, double *g_yz, double *g_occ)
{
    or_scene s0 = *s;
    s0.t_thr = 0.0f;
    or_sample *smp = (or_sample *)malloc(sizeof(or_sample) * (size_t)(s->n_max > 0 ? s->n_max : 1));
    double total = 0.0;
    for (long r = 0; r < n; r++) {
        or_march m;
        march_ray(&s0, rays + 6 * r, smp, &m);
        double S = 0.0;
        for (int i = 0; i < m.count; i++) S += smp[i].ah;
        if (!(S > 0.0)) continue;
        double L = 0.0;
        for (int i = 0; i < m.count; i++) {
            double p = smp[i].ah / S;
            if (p > 0.0) L -= p * log(p);
        }
        total += L;
        for (int i = 0; i < m.count; i++) {
            const or_sample *q = &smp[i];
            if (!(q->ah > 0.0)) continue;
            double da = grad_scale * lam / (double)n * (-(log(q->ah / S) + L) / S);
            double dsig = da * q->Mv * (1.0 - q->alpha);
            double dM = da * q->alpha;
            double dt[NCH] = {0, 0, 0, 0, 0, 0, 0, 0};
            dt[0] = dsig * q->sigma;
            or_stencil st;
            make_stencil(&s0, q->p, &st, NULL);
            scatter_stencil(&s0, &st, dt, g_grid, g_xy, g_xz, g_yz);
            if (g_occ) {
                if (q->branch == 1) g_occ[2 * q->cell] += dM * (-2.0 * q->r / (double)s->eps);
                if (q->branch == 2) g_occ[2 * q->cell + 1] += dM * (2.0 * q->r / (double)s->eps);
            }
        }
    }
    free(smp);
    return n > 0 ? lam * total / (double)n : 0.0;
}

/* ------------------------------------------------------------------ */
/* extraction after training (Sec. 4.4, Sec. 5.3)                      */
/* ------------------------------------------------------------------ */

/*
 * 3D occupancy grid of N[0] x N[1] x N[2] voxels over the box.  Voxel
 * (i, j, k) covers [x0 + i hx, x0 + (i + 1) hx) and the like; it is occupied
 * iff some point in it would be evaluated by the sample rule: an occupancy
 * cell overlapping its xy footprint (cells a with a/M < (i+1)/Nx and
 * (a+1)/M > i/Nx, integer arithmetic) has a non-empty interval with
 * z_min < z_hi and z_max > z_lo, where z_lo = z0 + k hz and z_hi = z0 +
 * (k + 1) hz, hz = (z1 - z0) / Nz, all in FP32 without fused operations.
 * out: one byte per voxel [Nx][Ny][Nz].  Returns the number occupied.
 */
long or_occupancy_grid(const float *aabb, const float *occ, int M, const int32_t *N, uint8_t *out)
{
    float hz = (aabb[5] - aabb[4]) / (float)N[2];
    long count = 0;
    for (long i = 0; i < N[0]; i++) {
        long alo = i * M / N[0], ahi = ((i + 1) * M + N[0] - 1) / N[0] - 1;
        for (long j = 0; j < N[1]; j++) {
            long blo = j * M / N[1], bhi = ((j + 1) * M + N[1] - 1) / N[1] - 1;
            for (long k = 0; k < N[2]; k++) {
                float zlo = aabb[4] + (float)k * hz;
                float zhi = aabb[4] + (float)(k + 1) * hz;
                int hit = 0;
                for (long a = alo; a <= ahi && !hit; a++)
                    for (long b = blo; b <= bhi && !hit; b++) {
                        float zmin = occ[2 * (a * M + b)], zmax = occ[2 * (a * M + b) + 1];
                        if (zmin < zmax && zmin < zhi && zmax > zlo) hit = 1;
                    }
                out[(i * N[1] + j) * N[2] + k] = (uint8_t)hit;
                count += hit;
            }
        }
    }
    return count;
}

/*
 * Brick pool [nb][B][B][B][8] of the bricks that `table` allocates, taken
 * from a dense grid [Lx][Ly][Lz][8] (src_table NULL) or from an older brick
 * pool with table src_table (same B).  Vertices beyond the grid, or in a
 * brick the source does not hold, are 0.
 */
void or_extract_bricks(const int32_t *L, int B, const int32_t *table, const float *src, const int32_t *src_table,
                       float *pool)
{
    int nb[3];
    for (int a = 0; a < 3; a++) nb[a] = (L[a] + B - 1) / B;
    for (long bi = 0; bi < nb[0]; bi++)
        for (long bj = 0; bj < nb[1]; bj++)
            for (long bk = 0; bk < nb[2]; bk++) {
                long t = (bi * nb[1] + bj) * nb[2] + bk;
                long b = table[t];
                if (b < 0) continue;
                for (long li = 0; li < B; li++)
                    for (long lj = 0; lj < B; lj++)
                        for (long lk = 0; lk < B; lk++) {
                            float *dst = pool + ((((b * B + li) * B + lj) * B) + lk) * NCH;
                            long i = bi * B + li, j = bj * B + lj, k = bk * B + lk;
                            const float *from = NULL;
                            if (i < L[0] && j < L[1] && k < L[2]) {
                                if (!src_table) {
                                    from = src + ((i * L[1] + j) * L[2] + k) * NCH;
                                } else if (src_table[t] >= 0) {
                                    from = src + ((((long)src_table[t] * B + li) * B + lj) * B + lk) * NCH;
                                }
                            }
                            for (int c = 0; c < NCH; c++) dst[c] = from ? from[c] : 0.0f;
                        }
            }
}

/*
 * Rows [k0, k1] of the XZ and YZ planes (Rz rows over the box's z-range)
 * that any evaluated sample can touch: samples lie strictly inside
 * (lo, hi), the occupancy hull (min z_min, max z_max over non-empty cells),
 * and the bilinear stencil reads rows floor(u) and floor(u) + 1 with u =
 * (z - z0) * ((Rz - 1) / (z1 - z0)) in FP32; one row of margin on each side.
 * zr = the cropped planes' z-range, z0 + k (z1 - z0) / (Rz - 1) in FP32.
 * Returns 0, or -1 when no cell is occupied.
 */
int or_plane_crop_rows(const float *aabb, int Rz, const float *occ, int M, int32_t rows[2], float zr[2])
{
    float lo = INFINITY, hi = -INFINITY;
    for (long c = 0; c < (long)M * M; c++) {
        float a = occ[2 * c], b = occ[2 * c + 1];
        if (!(a < b)) continue;
        if (a < lo) lo = a;
        if (b > hi) hi = b;
    }
    if (!(lo < hi)) return -1;
    float sc = (float)(Rz - 1) / (aabb[5] - aabb[4]);
    float ulo = (lo - aabb[4]) * sc, uhi = (hi - aabb[4]) * sc;
    long k0 = (long)floorf(ulo) - 1, k1 = (long)floorf(uhi) + 2;
    if (k0 < 0) k0 = 0;
    if (k1 > Rz - 1) k1 = Rz - 1;
    if (k0 > Rz - 2) k0 = Rz - 2;
    if (k1 < k0 + 1) k1 = k0 + 1;
    rows[0] = (int32_t)k0;
    rows[1] = (int32_t)k1;
    float h = (aabb[5] - aabb[4]) / (float)(Rz - 1);
    zr[0] = aabb[4] + (float)k0 * h;
    zr[1] = aabb[4] + (float)k1 * h;
    return 0;
}


/* ------------------------------------------------------------------ */
/* working set of a render (Sec. 4.4 viewer)                           */
/* ------------------------------------------------------------------ */
static void mark(uint8_t *m, long i)
{
    __atomic_store_n(&m[i], (uint8_t)1, __ATOMIC_RELAXED);
}

/* Marks every parameter a render of the rays reads at least once: the 8 grid
 * vertices (dense index or pool slot, over [vertices] = [Lx Ly Lz] or
 * [nb B^3]) and the 4 texels of each plane of every evaluated sample, and
 * the occupancy cell of every lattice sample inside the box that the march
 * tests before the ray stops.  Unallocated corners mark nothing.  Marks are
 * bytes set to 1; returns the number of evaluated samples. */
long or_working_set(const or_scene *s, const float *rays, long n, uint8_t *m_grid, uint8_t *m_xy, uint8_t *m_xz,
                    uint8_t *m_yz, uint8_t *m_occ, int nthreads)
{
    long samples = 0;
    const int nt = team_size(nthreads);
    uint8_t *planes[3] = {m_xy, m_xz, m_yz};
#pragma omp parallel num_threads(nt) reduction(+ : samples)
    {
        or_sample *smp = (or_sample *)malloc(sizeof(or_sample) * (size_t)(s->n_max > 0 ? s->n_max : 1));
#pragma omp for schedule(dynamic, 64)
        for (long r = 0; r < n; r++) {
            const float *ray = rays + 6 * r;
            or_march m;
            march_ray(s, ray, smp, &m);
            samples += m.count;
            for (int i = 0; i < m.count; i++) {
                or_stencil st;
                make_stencil(s, smp[i].p, &st, NULL);
                for (int c = 0; c < 8; c++)
                    if (st.gidx[c] >= 0) mark(m_grid, st.gidx[c] / NCH);
                for (int q = 0; q < 3; q++)
                    for (int t = 0; t < 4; t++) mark(planes[q], st.pidx[q][t] / NCH);
            }
            /* the candidates the march tests: all in-box lattice samples up
             * to the last evaluated one when the ray stopped early, else all */
            double tin, tout;
            if (!slab_range(s, ray, ray + 3, &tin, &tout)) continue;
            double fklo = floor(tin / s->step) - 2.0, fkhi = ceil(tout / s->step) + 2.0;
            if (fklo < 0.0) fklo = 0.0;
            if (fkhi > 16777215.0) fkhi = 16777215.0;
            int stopped = m.count > 0 && (m.count >= s->n_max || (s->t_thr > 0.0f && m.TN < (double)s->t_thr));
            long khi = stopped ? (long)m.k_last : (long)fkhi;
            for (long k = (long)fklo; k <= khi; k++) {
                float p[3];
                int cell = -1;
                lattice_test(s, ray, ray + 3, k, p, &cell);
                if (cell >= 0) mark(m_occ, cell);
            }
        }
        free(smp);
    }
    return samples;
}

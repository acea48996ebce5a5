/*
 * oracle.c -- plain, slow FP64 CPU oracle of the per-frame rendering path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this library.  It shares no code, header or
 * constant with the CUDA renderer; it reads the same FP32 scene arrays.
 *
 * What it computes, step by step, in the order of the paper's pipeline
 * (Sec. 3.1 "Pipeline": cut finding -> culling & projection -> sorting ->
 * rasterization), with the preemptive alpha filter of Sec. 4.2 (Eq. 3, 4):
 *
 *  1. Granularity test (the one FP32 formula; Sec. 3.1 "Cut Finding" gives
 *     only "projected size below tau, parent's above").  Projected size is
 *     f * R_n / |cam - c_n| in pixels, f = max(fx, fy).  With
 *     t = fl(tau / f), k = fl(t * t) and single-rounded FP32 operations:
 *        dx = cx - nx, dy = cy - ny, dz = cz - nz
 *        d2 = (dx*dx + dy*dy) + dz*dz
 *        expand(n) = n has children  and  fl(d2 * k) < radius2[n]
 *     (compiled with -ffp-contract=off: no FMA contraction).
 *  1b. Frustum-aware variant (the tree also "identifies the Gaussians inside
 *     the view frustum", Sec. 3.1; the paper gives no test, this is the
 *     reading used): expand(n) additionally needs n's axis-aligned box to
 *     meet five half-spaces.  In camera space their inward normals a and
 *     offsets o_c are: near (0,0,1), z_near; left (fx, 0, cx+g); right
 *     (-fx, 0, W-cx+g); top (0, fy, cy+g); bottom (0, -fy, H-cy+g); o_c = 0
 *     for the four sides (planes through the camera centre and the image
 *     edges moved out by g pixels).  World normal w = R^T a and offset
 *     o = w . C + o_c, computed in FP64 with correctly rounded fma in the
 *     order w_j = fma(R[2][j], a2, fma(R[1][j], a1, R[0][j] a0)), rounded to
 *     FP32, then o = fma(w2, C2, fma(w1, C1, w0 C0)) + o_c rounded to FP32.
 *     The box corner X furthest along w (hi where w_j >= 0, else lo) is
 *     tested: fl(fl(fl(w0 X0) + fl(w1 X1)) + fl(w2 X2)) - o >= 0.
 *  1c. Weight interpolation (Sec. 3.1 "Weight Interpolation": each cut
 *     Gaussian is interpolated with its parent; the paper gives no formula,
 *     this is the reading used).  With t = fl(tau / f) and a node's size
 *     ratio a = fl(sqrt(fl(radius2 / d2))) (d2 as in step 1, IEEE division
 *     and square root in FP32), the parent weight of cut node n with parent p
 *     is w = clamp(fl(fl(t - a_n) / fl(a_p - a_n)), 0, 1) when a_p > a_n and
 *     0 otherwise (and at the root): 0 where n is about to expand (a_n = t),
 *     1 where p is about to collapse (a_p = t).  The rendered Gaussian has the
 *     FP32 mean fl(m_n + fl(w fl(m_p - m_n))) per component (it decides the
 *     depth key, so both sides round it alike), and in FP64 the covariance
 *     S_n + w (S_p - S_n), the SH coefficients likewise, and the opacity
 *     theta_n + w (s_p - theta_n) with s_p = 1 - (1 - theta_p)^(1/k), k the
 *     number of children of p: the share of the parent's opacity that makes
 *     k coincident copies as opaque as the parent.
 *  2. Cut = { n : every strict ancestor expands and n does not }, found by a
 *     plain top-down traversal from the root.  A brute-force form (walk the
 *     ancestor chain of every node) is provided as a cross-check.
 *  3. Projection (EWA splatting conventions): p = R (mu - C) with R the
 *     world->camera rotation and C the camera centre; depth z = p_z; culled if
 *     z <= z_near.  u = fx x/z + cx, v = fy y/z + cy; pixel (i, j) has its
 *     centre at (i + 0.5, j + 0.5).  J = [[fx/z, 0, -fx tx/z], [0, fy/z,
 *     -fy ty/z]] with tx = clamp(x/z, +-1.3 (W/2)/fx), ty likewise;
 *     Sigma' = J R Sigma R^T J^T + 0.3 I; conic = Sigma'^-1 (culled if
 *     det <= 0).  Colour = sum_lm c_lm Y_lm(d) + 0.5 clamped at 0, with
 *     d = (mu - C)/|mu - C| and Y_lm the real orthonormal spherical
 *     harmonics (Condon-Shortley phase), evaluated from the associated
 *     Legendre recurrence.
 *  4. Preemptive alpha filter (Eq. 3, 4): alpha = min(0.99, theta e^rho) is
 *     at least alpha* = 1/255 iff rho >= ln alpha* - ln theta.  A Gaussian
 *     with theta < alpha* never reaches alpha* and is dropped.  Its footprint
 *     {rho >= ln alpha* - ln theta} has the exact bounding box
 *     u +- r sqrt(Sigma'_00), v +- r sqrt(Sigma'_11), r^2 = 2 (ln theta -
 *     ln alpha*).  A 16x16 tile is a candidate when the rectangle spanned by
 *     its pixel centres meets that box, and the pair is kept when the
 *     maximum of rho over that rectangle is >= ln alpha* - ln theta.
 *  5. Sort: kept pairs ordered by (tile, depth key, node id).  The depth key
 *     is the FP32 depth computed as ((R20*dx + R21*dy) + R22*dz) with
 *     dx = fl(mu_x - C_x) ..., single-rounded; the near-plane decision also
 *     uses it.  Discrete decisions (order, near cull) are thus taken in the
 *     renderer's precision; everything continuous is FP64.
 *  6. Blend front to back per pixel (Sec. 3.1 "Rasterization", Eq. 3):
 *     rho = -1/2 (a dx^2 + c dy^2) - b dx dy, alpha = min(0.99, theta e^rho);
 *     skip when alpha < alpha*; T' = T (1 - alpha); stop (without this
 *     Gaussian) when T' < 1e-4; else C += alpha T rgb, T = T'.  Background 0.
 *  6b. Lookup-table variant (Sec. 4.2, Eq. 5), selected by m = lut_m > 0:
 *     the alpha* decision is Eq. 4's (skip when rho < ln alpha* - ln theta),
 *     then e^rho is replaced by the nearest of the m + 1 samples
 *     e^(-5.55 i / m), i = 0..m, of the effective range [-5.55, 0]:
 *     i = round(rho / -5.55 * m) to nearest, ties to even, clamped to
 *     [0, m]; alpha = min(0.99, theta e^(-5.55 i / m)) with no second alpha*
 *     test.  The index is an integer decided by floating point, so it is
 *     taken in the renderer's precision: fl(fl(rho) * fl(-fl(m) / 5.55f)).
 *     The rest of step 6 is unchanged.
 *  7. Exhaustive mode: the same per-pixel loop over every cut Gaussian that
 *     passes the near-plane and determinant culls, sorted by (depth key,
 *     id), with no tiles, boxes or filters.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    uint32_t n_nodes, sh_degree;
    const uint32_t* parent;      /* root: 0xFFFFFFFF */
    const uint32_t* first_child;
    const uint8_t* n_child;
    const float* mean;           /* 3N */
    const float* cov6;           /* 6N: xx xy xz yy yz zz */
    const float* opacity;        /* N */
    const float* sh;             /* N * (deg+1)^2 * 3, coefficient-major */
    const float* radius2;        /* N */
    const float* bbox;           /* 6N: lo xyz, hi xyz (frustum-aware variant only) */
} orc_scene;

typedef struct {
    float R[9];                  /* world -> camera rotation, row-major */
    float pos[3];                /* camera centre C in world coordinates */
    float fx, fy, cx, cy;
    uint32_t width, height;
    float z_near;
} orc_camera;

#define ORC_TILE 16  /* the default tile size (pixels per side) */
static const double ORC_ALPHA_MIN = 1.0 / 255.0;
static const double ORC_T_MIN = 1e-4;
static const double ORC_ALPHA_MAX = 0.99;
static const double ORC_DILATE = 0.3;
static const double ORC_PI = 3.14159265358979323846264338327950288;

/* --------------------------------------------------- 1. granularity test */
float orc_lod_k(float tau, float f) {
    float t = tau / f;
    return t * t;
}

/* t = fl(tau / f), the size ratio of the granularity threshold */
static float orc_lod_k_t(float tau, float f) { return tau / f; }

/* 1b: the five planes as (w0, w1, w2, o) in planes[4 i ..] */
void orc_frustum_planes(const orc_camera* cam, float guard, float planes[20]) {
    double g = guard, W = cam->width, H = cam->height;
    double a[5][3] = {{0.0, 0.0, 1.0},
                      {cam->fx, 0.0, (double)cam->cx + g},
                      {-(double)cam->fx, 0.0, (W - cam->cx) + g},
                      {0.0, cam->fy, (double)cam->cy + g},
                      {0.0, -(double)cam->fy, (H - cam->cy) + g}};
    double oc[5] = {cam->z_near, 0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < 5; ++i) {
        float w[3];
        for (int j = 0; j < 3; ++j) {
            /* (R^T a)_j = sum over camera axes r of R[r][j] a_r */
            double acc = (double)cam->R[0 * 3 + j] * a[i][0];
            acc = fma((double)cam->R[1 * 3 + j], a[i][1], acc);
            acc = fma((double)cam->R[2 * 3 + j], a[i][2], acc);
            w[j] = (float)acc;
        }
        double o = (double)w[0] * (double)cam->pos[0];
        o = fma((double)w[1], (double)cam->pos[1], o);
        o = fma((double)w[2], (double)cam->pos[2], o);
        planes[4 * i + 0] = w[0];
        planes[4 * i + 1] = w[1];
        planes[4 * i + 2] = w[2];
        planes[4 * i + 3] = (float)(o + oc[i]);
    }
}

/* 1b: does the box lo[3], hi[3] meet every half-space w . x - o >= 0? */
int orc_box_meets(const float box[6], const float planes[20]) {
    for (int i = 0; i < 5; ++i) {
        const float* p = planes + 4 * i;
        float X = p[0] >= 0.0f ? box[3] : box[0];
        float Y = p[1] >= 0.0f ? box[4] : box[1];
        float Z = p[2] >= 0.0f ? box[5] : box[2];
        float t0 = p[0] * X, t1 = p[1] * Y, t2 = p[2] * Z;
        float sum = (t0 + t1) + t2;
        float sd = sum - p[3];
        if (!(sd >= 0.0f)) return 0;
    }
    return 1;
}

/* planes == NULL: the distance test of step 1 alone; else also step 1b */
static int orc_expand(const orc_scene* s, uint32_t n, const float cam[3], float k, const float* planes) {
    if (s->n_child[n] == 0) return 0;
    float dx = cam[0] - s->mean[3 * (size_t)n + 0];
    float dy = cam[1] - s->mean[3 * (size_t)n + 1];
    float dz = cam[2] - s->mean[3 * (size_t)n + 2];
    float d2 = (dx * dx + dy * dy) + dz * dz;
    float lhs = d2 * k;
    if (!(lhs < s->radius2[n])) return 0;
    return planes ? orc_box_meets(s->bbox + 6 * (size_t)n, planes) : 1;
}

int orc_expand_node(const orc_scene* s, uint32_t n, const float cam[3], float k, const float* planes) {
    return orc_expand(s, n, cam, k, planes);
}

static int orc_cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------ 2. the cut */
/* Top-down traversal from the root; out must hold n_nodes ids; returns |C|
 * with the ids in ascending order. */
int64_t orc_cut_topdown(const orc_scene* s, const float cam[3], float k, const float* planes, uint32_t* out) {
    if (s->n_nodes == 0) return 0;
    uint32_t* stack = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)s->n_nodes);
    if (!stack) return -1;
    int64_t sp = 0, nc = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        uint32_t n = stack[--sp];
        if (orc_expand(s, n, cam, k, planes)) {
            for (uint32_t c = 0; c < s->n_child[n]; ++c) stack[sp++] = s->first_child[n] + c;
        } else {
            out[nc++] = n;
        }
    }
    free(stack);
    qsort(out, (size_t)nc, sizeof(uint32_t), orc_cmp_u32);
    return nc;
}

/* The definition read literally: n is in the cut iff it does not expand and
 * every node on its ancestor chain does. */
int64_t orc_cut_bruteforce(const orc_scene* s, const float cam[3], float k, const float* planes, uint32_t* out) {
    int64_t nc = 0;
    for (uint32_t n = 0; n < s->n_nodes; ++n) {
        if (orc_expand(s, n, cam, k, planes)) continue;
        int ok = 1;
        for (uint32_t a = s->parent[n]; a != 0xFFFFFFFFu; a = s->parent[a])
            if (!orc_expand(s, a, cam, k, planes)) { ok = 0; break; }
        if (ok) out[nc++] = n;
    }
    return nc;
}

/* ------------------------------------------------- spherical harmonics */
/* Real orthonormal SH up to degree 3, index l*l + l + m, from
 *   Y_l0 = K_l0 P_l^0(cos t)
 *   Y_lm = sqrt2 K_lm P_l^m(cos t) cos(m phi)        (m > 0)
 *   Y_lm = sqrt2 K_l|m| P_l^|m|(cos t) sin(|m| phi)  (m < 0)
 *   K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)
 * with P_l^m including the Condon-Shortley phase (-1)^m. */
static double orc_fact(int n) { double r = 1.0; for (int i = 2; i <= n; ++i) r *= i; return r; }

static double orc_legendre(int l, int m, double x) {
    /* P_m^m = (-1)^m (2m-1)!! (1-x^2)^(m/2) */
    double pmm = 1.0;
    double sx = sqrt(fmax(0.0, 1.0 - x * x));
    for (int i = 1; i <= m; ++i) pmm *= -(2.0 * i - 1.0) * sx;
    if (l == m) return pmm;
    double pm1 = x * (2.0 * m + 1.0) * pmm; /* P_{m+1}^m */
    if (l == m + 1) return pm1;
    double pl = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        pl = ((2.0 * ll - 1.0) * x * pm1 - (ll + m - 1.0) * pmm) / (ll - m);
        pmm = pm1;
        pm1 = pl;
    }
    return pl;
}

void orc_sh_basis(int degree, const double d[3], double* Y) {
    double ct = d[2];
    double phi = atan2(d[1], d[0]);
    for (int l = 0; l <= degree; ++l)
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI) * orc_fact(l - am) / orc_fact(l + am));
            double P = orc_legendre(l, am, ct);
            double v;
            if (m == 0) v = K * P;
            else if (m > 0) v = sqrt(2.0) * K * P * cos(m * phi);
            else v = sqrt(2.0) * K * P * sin(am * phi);
            Y[l * l + l + m] = v;
        }
}

/* ------------------------------------------------------- 3. projection */
typedef struct {
    int32_t valid;       /* passed near-plane and determinant culls */
    int32_t visible;     /* has at least one kept tile */
    float zkey;          /* FP32 depth key */
    double z;            /* FP64 depth */
    double u, v;         /* projected mean, pixels */
    double cov[3];       /* Sigma' (00, 01, 11) incl. dilation */
    double conic[3];     /* a, b, c */
    double rgb[3];
    double theta;        /* opacity */
    double thr;          /* ln alpha* - ln theta */
    int32_t rect[4];     /* candidate tiles: tx0, ty0, tx1, ty1 (inclusive), empty if tx0 > tx1 */
    int32_t ntile;       /* kept tiles */
} orc_proj;

/* 1c: a node's size ratio R / d in FP32 */
static float orc_size_ratio(const orc_scene* s, uint32_t n, const float cam[3]) {
    float dx = cam[0] - s->mean[3 * (size_t)n + 0];
    float dy = cam[1] - s->mean[3 * (size_t)n + 1];
    float dz = cam[2] - s->mean[3 * (size_t)n + 2];
    float d2 = (dx * dx + dy * dy) + dz * dz;
    float q = s->radius2[n] / d2;
    return sqrtf(q);
}

/* 1c: parent weight of cut node n (0 at the root) */
float orc_interp_weight(const orc_scene* s, uint32_t n, const float cam[3], float t) {
    uint32_t p = s->parent[n];
    if (p == 0xFFFFFFFFu) return 0.0f;
    float an = orc_size_ratio(s, n, cam), ap = orc_size_ratio(s, p, cam);
    if (!(ap > an)) return 0.0f;
    float num = t - an, den = ap - an;
    float w = num / den;
    return fminf(1.0f, fmaxf(0.0f, w));
}

/* interp_t < 0: the node's own Gaussian; else step 1c with t = interp_t */
static void orc_project_one(const orc_scene* s, const orc_camera* cam, uint32_t n, orc_proj* P, float interp_t) {
    memset(P, 0, sizeof(*P));
    P->rect[0] = 0; P->rect[1] = 0; P->rect[2] = -1; P->rect[3] = -1;
    int deg = (int)s->sh_degree;
    int K = (deg + 1) * (deg + 1);
    float mf[3];
    double c6[6], theta_n, shn[48];
    for (int j = 0; j < 3; ++j) mf[j] = s->mean[3 * (size_t)n + j];
    for (int j = 0; j < 6; ++j) c6[j] = s->cov6[6 * (size_t)n + j];
    theta_n = s->opacity[n];
    for (int j = 0; j < 3 * K; ++j) shn[j] = s->sh[(size_t)n * K * 3 + j];
    if (interp_t >= 0.0f) {
        float w = orc_interp_weight(s, n, cam->pos, interp_t);
        if (w > 0.0f) {
            uint32_t p = s->parent[n];
            for (int j = 0; j < 3; ++j) {
                float dm = s->mean[3 * (size_t)p + j] - mf[j];
                float wd = w * dm;
                mf[j] = mf[j] + wd;
            }
            double wd = w;
            for (int j = 0; j < 6; ++j) c6[j] += wd * ((double)s->cov6[6 * (size_t)p + j] - c6[j]);
            double share = -expm1(log1p(-(double)s->opacity[p]) / (double)s->n_child[p]);
            theta_n += wd * (share - theta_n);
            for (int j = 0; j < 3 * K; ++j) shn[j] += wd * ((double)s->sh[(size_t)p * K * 3 + j] - shn[j]);
        }
    }
    /* depth key: the renderer's FP32 expression */
    float dxf = mf[0] - cam->pos[0], dyf = mf[1] - cam->pos[1], dzf = mf[2] - cam->pos[2];
    float zk = (cam->R[6] * dxf + cam->R[7] * dyf) + cam->R[8] * dzf;
    P->zkey = zk;
    if (!(zk > cam->z_near)) return;

    double d[3] = {(double)mf[0] - cam->pos[0], (double)mf[1] - cam->pos[1], (double)mf[2] - cam->pos[2]};
    double R[9];
    for (int i = 0; i < 9; ++i) R[i] = cam->R[i];
    double p[3];
    for (int r = 0; r < 3; ++r) p[r] = R[3 * r] * d[0] + R[3 * r + 1] * d[1] + R[3 * r + 2] * d[2];
    double z = p[2];
    P->z = z;
    double fx = cam->fx, fy = cam->fy;
    P->u = fx * p[0] / z + cam->cx;
    P->v = fy * p[1] / z + cam->cy;

    double S[9] = {c6[0], c6[1], c6[2], c6[1], c6[3], c6[4], c6[2], c6[4], c6[5]};
    double RS[9], Sc[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += R[3 * r + k] * S[3 * k + c];
            RS[3 * r + c] = acc;
        }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += RS[3 * r + k] * R[3 * c + k];
            Sc[3 * r + c] = acc;
        }
    double limx = 1.3 * (0.5 * (double)cam->width / fx);
    double limy = 1.3 * (0.5 * (double)cam->height / fy);
    double tx = fmin(limx, fmax(-limx, p[0] / z));
    double ty = fmin(limy, fmax(-limy, p[1] / z));
    double J[6] = {fx / z, 0.0, -fx * tx / z, 0.0, fy / z, -fy * ty / z};
    double JS[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += J[3 * r + k] * Sc[3 * k + c];
            JS[3 * r + c] = acc;
        }
    double C2[4];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += JS[3 * r + k] * J[3 * c + k];
            C2[2 * r + c] = acc;
        }
    double s00 = C2[0] + ORC_DILATE, s01 = 0.5 * (C2[1] + C2[2]), s11 = C2[3] + ORC_DILATE;
    P->cov[0] = s00; P->cov[1] = s01; P->cov[2] = s11;
    double det = s00 * s11 - s01 * s01;
    if (!(det > 0.0)) return;
    P->conic[0] = s11 / det;
    P->conic[1] = -s01 / det;
    P->conic[2] = s00 / det;
    P->valid = 1;

    /* colour */
    double nd = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double dir[3] = {d[0] / nd, d[1] / nd, d[2] / nd};
    double Y[16];
    orc_sh_basis(deg, dir, Y);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) acc += shn[3 * k + ch] * Y[k];
        acc += 0.5;
        P->rgb[ch] = acc > 0.0 ? acc : 0.0;
    }
    P->theta = theta_n;
    P->thr = log(ORC_ALPHA_MIN) - log(P->theta > 0.0 ? P->theta : 1e-300);
}

/* ---------------------------------------------------- 4. tile filtering */
static double orc_rho(const double conic[3], double dx, double dy) {
    return -0.5 * (conic[0] * dx * dx + conic[2] * dy * dy) - conic[1] * dx * dy;
}

static double orc_clamp(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* max of rho over [x0,x1] x [y0,y1] (pixel-centre rectangle) */
double orc_rho_max_rect(const double conic[3], double u, double v, double x0, double x1, double y0,
                        double y1) {
    if (u >= x0 && u <= x1 && v >= y0 && v <= y1) return 0.0;
    double a = conic[0], b = conic[1], c = conic[2];
    double best = -INFINITY;
    double xs[2] = {x0, x1}, ys[2] = {y0, y1};
    for (int e = 0; e < 2; ++e) {
        double dx = xs[e] - u; /* vertical edge: dx fixed, dy free */
        double dy = orc_clamp(-b * dx / c, y0 - v, y1 - v);
        double r = orc_rho(conic, dx, dy);
        if (r > best) best = r;
        double dy2 = ys[e] - v; /* horizontal edge: dy fixed, dx free */
        double dx2 = orc_clamp(-b * dy2 / a, x0 - u, x1 - u);
        r = orc_rho(conic, dx2, dy2);
        if (r > best) best = r;
    }
    return best;
}

/* pixel-centre rectangle of tile (tx, ty), tiles of tile x tile pixels */
static void orc_tile_rect(const orc_camera* cam, int tile, int tx, int ty, double* x0, double* x1, double* y0,
                          double* y1) {
    *x0 = tile * tx + 0.5;
    *x1 = fmin(tile * tx + tile - 0.5, (double)cam->width - 0.5);
    *y0 = tile * ty + 0.5;
    *y1 = fmin(tile * ty + tile - 0.5, (double)cam->height - 0.5);
}

/* candidate tile rectangle from the opacity-aware bounding box */
static void orc_candidates(const orc_camera* cam, int tile, orc_proj* P) {
    P->rect[0] = 0; P->rect[1] = 0; P->rect[2] = -1; P->rect[3] = -1;
    if (!P->valid) return;
    if (P->theta < ORC_ALPHA_MIN) return; /* Gaussian-level filter */
    double r2 = 2.0 * (log(P->theta) - log(ORC_ALPHA_MIN));
    if (r2 < 0.0) r2 = 0.0;
    double bx = sqrt(r2 * P->cov[0]), by = sqrt(r2 * P->cov[2]);
    int TW = (int)((cam->width + tile - 1) / tile), TH = (int)((cam->height + tile - 1) / tile);
    double fx0 = ceil((P->u - bx - (tile - 0.5)) / tile);
    double fx1 = floor((P->u + bx - 0.5) / tile);
    double fy0 = ceil((P->v - by - (tile - 0.5)) / tile);
    double fy1 = floor((P->v + by - 0.5) / tile);
    fx0 = fmax(fx0, 0.0); fy0 = fmax(fy0, 0.0);
    fx1 = fmin(fx1, TW - 1.0); fy1 = fmin(fy1, TH - 1.0);
    if (fx0 > fx1 || fy0 > fy1) return;
    P->rect[0] = (int32_t)fx0; P->rect[1] = (int32_t)fy0;
    P->rect[2] = (int32_t)fx1; P->rect[3] = (int32_t)fy1;
}

/* ------------------------------------------------------------- results */
typedef struct {
    int64_t n_cut;
    uint32_t* cut;            /* ascending node ids */
    orc_proj* proj;           /* per cut entry */
    /* candidate pairs (tile, cut index) with margin rho_max - thr */
    int64_t n_cand;
    uint32_t* cand_tile;
    uint32_t* cand_idx;
    double* cand_margin;
    int64_t n_pairs;          /* kept pairs in render order */
    uint32_t* pair_tile;
    uint32_t* pair_idx;
    int64_t* tile_start;      /* n_tiles + 1 */
    int64_t n_tiles;
    double* image;            /* H x W x 3 */
    uint8_t* flags;           /* H x W: 1 = near an alpha* or T_min boundary */
    uint32_t* n_eval;         /* H x W: evaluated pairs */
    uint32_t* n_contrib;      /* H x W: blended Gaussians */
    int64_t n_visible;
    int64_t n_eval_total;
} orc_frame;

void orc_frame_free(orc_frame* f) {
    if (!f) return;
    free(f->cut); free(f->proj); free(f->cand_tile); free(f->cand_idx); free(f->cand_margin);
    free(f->pair_tile); free(f->pair_idx); free(f->tile_start); free(f->image); free(f->flags);
    free(f->n_eval); free(f->n_contrib); free(f);
}

typedef struct {
    uint32_t tile;
    float zkey;
    uint32_t node;
    uint32_t idx;
} orc_key;

static int orc_cmp_key(const void* a, const void* b) {
    const orc_key* x = (const orc_key*)a;
    const orc_key* y = (const orc_key*)b;
    if (x->tile != y->tile) return x->tile < y->tile ? -1 : 1;
    if (x->zkey != y->zkey) return x->zkey < y->zkey ? -1 : 1;
    if (x->node != y->node) return x->node < y->node ? -1 : 1;
    return 0;
}

/* Per-pixel front-to-back blend over the list idx[0..n).  The ambiguity
 * flag marks pixels where a renderer working in FP32 may legitimately take
 * the other side of the alpha >= alpha* decision for some Gaussian (rho within
 * 'band' of ln alpha* - ln theta) while the transmittance is still at least
 * t_flag, so that the flip could move the pixel by up to about
 * alpha* T max(rgb).  Flips of the T < 1e-4 test move a pixel by at most
 * about 1e-4 max(rgb) and are not flagged. */
static void orc_blend_pixel(const orc_proj* P, const uint32_t* idx, int64_t n, double px, double py,
                            double band, double t_flag, uint32_t lut_m, double* out, uint8_t* flag,
                            uint32_t* n_eval, uint32_t* n_contrib) {
    const float lut_scale = lut_m ? -(float)lut_m / 5.55f : 0.0f;
    double T = 1.0, C[3] = {0, 0, 0};
    uint8_t f = 0;
    uint32_t ne = 0, nb = 0;
    for (int64_t i = 0; i < n; ++i) {
        const orc_proj* g = &P[idx[i]];
        double dx = g->u - px, dy = g->v - py;
        double rho = orc_rho(g->conic, dx, dy);
        ++ne;
        if (fabs(rho - g->thr) <= band && T >= t_flag) f = 1;
        double alpha;
        if (lut_m) {
            if (rho < g->thr) continue; /* Eq. 4 */
            float q = nearbyintf((float)rho * lut_scale);
            uint32_t i = q <= 0.0f ? 0u : (q >= (float)lut_m ? lut_m : (uint32_t)q);
            alpha = fmin(ORC_ALPHA_MAX, g->theta * exp(-5.55 * (double)i / (double)lut_m));
        } else {
            alpha = fmin(ORC_ALPHA_MAX, g->theta * exp(rho));
            if (alpha < ORC_ALPHA_MIN) continue;
        }
        double Tn = T * (1.0 - alpha);
        if (Tn < ORC_T_MIN) break;
        for (int ch = 0; ch < 3; ++ch) C[ch] += alpha * T * g->rgb[ch];
        T = Tn;
        ++nb;
    }
    out[0] = C[0]; out[1] = C[1]; out[2] = C[2];
    *flag = f;
    *n_eval = ne;
    *n_contrib = nb;
}

/*
 * Render one frame.  tile_mask (optional, n_tiles bytes) restricts binning
 * and blending to the flagged tiles.  band and t_flag parameterise the
 * ambiguity flag (see orc_blend_pixel).  exhaustive != 0 selects mode 7.
 * frustum_guard >= 0 (with s->bbox) selects the frustum-aware cut (1b);
 * interp != 0 renders the cut's Gaussians interpolated with their parents (1c).
 * lut_m > 0 blends with the Eq. 5 lookup table of m intervals (6b).
 * tile: the side of a square tile in pixels (0: ORC_TILE); tile_mask and the
 * pair lists are per tile of that size.  Binning is exact whatever the size
 * (no pixel with alpha >= alpha* lies outside a kept pair), so the image does
 * not depend on it.
 */
orc_frame* orc_render(const orc_scene* s, const orc_camera* cam, float tau, const uint8_t* tile_mask,
                      double band, double t_flag, int exhaustive, float frustum_guard, int interp,
                      uint32_t lut_m, uint32_t tile_px) {
    const int tile = tile_px ? (int)tile_px : ORC_TILE;
    orc_frame* F = (orc_frame*)calloc(1, sizeof(orc_frame));
    if (!F) return NULL;
    float f = cam->fx > cam->fy ? cam->fx : cam->fy;
    float k = orc_lod_k(tau, f);
    F->cut = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(s->n_nodes ? s->n_nodes : 1));
    if (!F->cut) { orc_frame_free(F); return NULL; }
    float planes[20];
    const int frustum = frustum_guard >= 0.0f && s->bbox;  /* step 1b when a guard is given */
    if (frustum) orc_frustum_planes(cam, frustum_guard, planes);
    F->n_cut = orc_cut_topdown(s, cam->pos, k, frustum ? planes : NULL, F->cut);
    if (F->n_cut < 0) { orc_frame_free(F); return NULL; }
    int64_t nc = F->n_cut;
    F->proj = (orc_proj*)calloc((size_t)(nc ? nc : 1), sizeof(orc_proj));
    if (!F->proj) { orc_frame_free(F); return NULL; }
    int64_t i;
#pragma omp parallel for schedule(dynamic, 256)
    for (i = 0; i < nc; ++i) {
        orc_project_one(s, cam, F->cut[i], &F->proj[i], interp ? orc_lod_k_t(tau, f) : -1.0f);
        orc_candidates(cam, tile, &F->proj[i]);
    }
    const int W = (int)cam->width, H = (int)cam->height;
    const int TW = (W + tile - 1) / tile, TH = (H + tile - 1) / tile;
    F->n_tiles = (int64_t)TW * TH;
    size_t npx = (size_t)W * H;
    F->image = (double*)calloc(npx ? npx * 3 : 1, sizeof(double));
    F->flags = (uint8_t*)calloc(npx ? npx : 1, 1);
    F->n_eval = (uint32_t*)calloc(npx ? npx : 1, sizeof(uint32_t));
    F->n_contrib = (uint32_t*)calloc(npx ? npx : 1, sizeof(uint32_t));
    F->tile_start = (int64_t*)calloc((size_t)F->n_tiles + 1, sizeof(int64_t));
    if (!F->image || !F->flags || !F->n_eval || !F->n_contrib || !F->tile_start) {
        orc_frame_free(F); return NULL;
    }

    if (exhaustive) {
        /* every near/det-surviving cut Gaussian, ordered by (depth key, id) */
        orc_key* keys = (orc_key*)malloc(sizeof(orc_key) * (size_t)(nc ? nc : 1));
        uint32_t* list = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(nc ? nc : 1));
        if (!keys || !list) { free(keys); free(list); orc_frame_free(F); return NULL; }
        int64_t m = 0;
        for (int64_t g = 0; g < nc; ++g)
            if (F->proj[g].valid) {
                keys[m].tile = 0; keys[m].zkey = F->proj[g].zkey; keys[m].node = F->cut[g];
                keys[m].idx = (uint32_t)g; ++m;
            }
        qsort(keys, (size_t)m, sizeof(orc_key), orc_cmp_key);
        for (int64_t g = 0; g < m; ++g) list[g] = keys[g].idx;
        free(keys);
        int64_t p;
#pragma omp parallel for schedule(dynamic, 64)
        for (p = 0; p < (int64_t)npx; ++p) {
            int x = (int)(p % W), y = (int)(p / W);
            int t = (y / tile) * TW + x / tile;
            if (tile_mask && !tile_mask[t]) continue;
            orc_blend_pixel(F->proj, list, m, x + 0.5, y + 0.5, band, t_flag, lut_m, &F->image[3 * p],
                            &F->flags[p], &F->n_eval[p], &F->n_contrib[p]);
        }
        free(list);
        int64_t tot = 0;
        for (p = 0; p < (int64_t)npx; ++p) tot += F->n_eval[p];
        F->n_eval_total = tot;
        return F;
    }

    /* candidates: count, prefix, fill (ordered by cut index, then tile) */
    int64_t* ccount = (int64_t*)calloc((size_t)nc + 1, sizeof(int64_t));
    if (!ccount) { orc_frame_free(F); return NULL; }
#pragma omp parallel for schedule(dynamic, 256)
    for (i = 0; i < nc; ++i) {
        const orc_proj* P = &F->proj[i];
        int64_t c = 0;
        for (int ty = P->rect[1]; ty <= P->rect[3]; ++ty)
            for (int tx = P->rect[0]; tx <= P->rect[2]; ++tx)
                if (!tile_mask || tile_mask[ty * TW + tx]) ++c;
        ccount[i + 1] = c;
    }
    for (i = 0; i < nc; ++i) ccount[i + 1] += ccount[i];
    F->n_cand = ccount[nc];
    size_t ncd = (size_t)(F->n_cand ? F->n_cand : 1);
    F->cand_tile = (uint32_t*)malloc(sizeof(uint32_t) * ncd);
    F->cand_idx = (uint32_t*)malloc(sizeof(uint32_t) * ncd);
    F->cand_margin = (double*)malloc(sizeof(double) * ncd);
    if (!F->cand_tile || !F->cand_idx || !F->cand_margin) { free(ccount); orc_frame_free(F); return NULL; }
#pragma omp parallel for schedule(dynamic, 256)
    for (i = 0; i < nc; ++i) {
        orc_proj* P = &F->proj[i];
        int64_t o = ccount[i];
        int32_t kept = 0;
        for (int ty = P->rect[1]; ty <= P->rect[3]; ++ty)
            for (int tx = P->rect[0]; tx <= P->rect[2]; ++tx) {
                if (tile_mask && !tile_mask[ty * TW + tx]) continue;
                double x0, x1, y0, y1;
                orc_tile_rect(cam, tile, tx, ty, &x0, &x1, &y0, &y1);
                double rm = orc_rho_max_rect(P->conic, P->u, P->v, x0, x1, y0, y1);
                F->cand_tile[o] = (uint32_t)(ty * TW + tx);
                F->cand_idx[o] = (uint32_t)i;
                F->cand_margin[o] = rm - P->thr;
                if (rm >= P->thr) ++kept;
                ++o;
            }
        P->ntile = kept;
        P->visible = kept > 0;
    }
    free(ccount);
    int64_t nv = 0, np = 0;
    for (i = 0; i < nc; ++i) { nv += F->proj[i].visible; np += F->proj[i].ntile; }
    F->n_visible = nv;
    F->n_pairs = np;

    /* kept pairs sorted by (tile, depth key, node id) */
    orc_key* keys = (orc_key*)malloc(sizeof(orc_key) * (size_t)(np ? np : 1));
    F->pair_tile = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(np ? np : 1));
    F->pair_idx = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(np ? np : 1));
    if (!keys || !F->pair_tile || !F->pair_idx) { free(keys); orc_frame_free(F); return NULL; }
    int64_t q = 0;
    for (int64_t c = 0; c < F->n_cand; ++c)
        if (F->cand_margin[c] >= 0.0) {
            uint32_t g = F->cand_idx[c];
            keys[q].tile = F->cand_tile[c]; keys[q].zkey = F->proj[g].zkey;
            keys[q].node = F->cut[g]; keys[q].idx = g; ++q;
        }
    qsort(keys, (size_t)np, sizeof(orc_key), orc_cmp_key);
    for (q = 0; q < np; ++q) { F->pair_tile[q] = keys[q].tile; F->pair_idx[q] = keys[q].idx; }
    free(keys);
    for (q = 0; q < np; ++q) F->tile_start[F->pair_tile[q] + 1]++;
    for (int64_t t = 0; t < F->n_tiles; ++t) F->tile_start[t + 1] += F->tile_start[t];

    /* blend per tile */
    int64_t t;
#pragma omp parallel for schedule(dynamic, 1)
    for (t = 0; t < F->n_tiles; ++t) {
        if (tile_mask && !tile_mask[t]) continue;
        int tx = (int)(t % TW), ty = (int)(t / TW);
        const uint32_t* list = F->pair_idx + F->tile_start[t];
        int64_t n = F->tile_start[t + 1] - F->tile_start[t];
        for (int y = ty * tile; y < (ty + 1) * tile && y < H; ++y)
            for (int x = tx * tile; x < (tx + 1) * tile && x < W; ++x) {
                size_t p = (size_t)y * W + x;
                orc_blend_pixel(F->proj, list, n, x + 0.5, y + 0.5, band, t_flag, lut_m, &F->image[3 * p],
                                &F->flags[p], &F->n_eval[p], &F->n_contrib[p]);
            }
    }
    int64_t tot = 0;
    for (size_t p = 0; p < npx; ++p) tot += F->n_eval[p];
    F->n_eval_total = tot;
    return F;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

size_t orc_proj_size(void) { return sizeof(orc_proj); }
size_t orc_frame_size(void) { return sizeof(orc_frame); }

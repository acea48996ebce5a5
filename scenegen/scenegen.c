/*
 * scenegen.c -- seeded synthetic Gaussian scenes and their LoD tree.
 *
 * Input infrastructure shared by the CPU oracle tests and the GPU renderer
 * tests/bench.  It holds none of the per-frame method (no cut finding, no
 * projection, no sorting, no blending): it only draws leaf Gaussians and
 * builds the LoD tree the method consumes (one Gaussian per node, variable
 * fan-out, finer Gaussians on lower levels; paper Sec. 3.1 "LoD Tree").
 *
 * Random numbers: counter-based SplitMix64.  Draw j of item i is
 *     mix64(key + (i*256 + j + 1) * 0x9E3779B97F4A7C15)
 * with key = mix64(seed).  Results therefore do not depend on the thread
 * count.  Normals come from Box-Muller in FP64.
 *
 * Tree: leaves are sorted by 63-bit Morton code (21 bits per axis over the
 * bounding cube of the means, ties by leaf index); a node splits its range
 * by the highest 3-bit Morton digit that is not constant over the range
 * (so single-child chains are collapsed); ranges whose codes are all equal
 * are split into <= 8 contiguous chunks.  Nodes are numbered breadth-first,
 * node 0 is the root, the children of a node are contiguous and every child
 * id is larger than its parent id.
 *
 * Parents are the opacity-weighted moment-matched merge of their children
 * (weights w_i = opacity_i):
 *     mu_p  = sum w_i mu_i / W
 *     Sig_p = sum w_i (Sig_i + (mu_i - mu_p)(mu_i - mu_p)^T) / W
 *     SH_p  = sum w_i SH_i / W
 *     op_p  = min(0.99, 1 - prod(1 - op_i))
 * Radii nest: R_leaf = 3 * max axis scale, and
 *     R_p = (1 + 2^-12) * max_i(|mu_p - mu_i| + R_i)
 * evaluated in FP64 from the stored FP32 values; radius2 is R^2 rounded up
 * to FP32.  This nesting keeps "child expands => parent expands" true for a
 * distance/size granularity test whenever tau <= focal length.
 *
 * Node boxes (for the frustum-aware variant of the granularity test): the
 * axis-aligned box of a node holds its own Gaussian's extent mu_j +- 3.34
 * sqrt(Sigma_jj) (FP64 from the stored FP32 values, rounded outward to FP32)
 * and the boxes of its children, so boxes nest exactly.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no fast-math, so
 * x86-64 and aarch64 builds give the same numbers up to libm last-ulp).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ RNG */
static inline uint64_t sg_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static inline uint64_t sg_bits(uint64_t key, uint64_t i, uint32_t j) {
    return sg_mix64(key + (i * 256ull + (uint64_t)j + 1ull) * 0x9E3779B97F4A7C15ull);
}
/* uniform in [0, 1) with 53 random bits */
static inline double sg_unif(uint64_t key, uint64_t i, uint32_t j) {
    return (double)(sg_bits(key, i, j) >> 11) * 0x1p-53;
}
/* m-th standard normal of item i: Box-Muller over uniforms 64+2*(m/2), +1 */
static inline double sg_normal(uint64_t key, uint64_t i, uint32_t m) {
    uint32_t j = 64u + 2u * (m >> 1);
    double u1 = 1.0 - sg_unif(key, i, j); /* (0, 1] */
    double u2 = sg_unif(key, i, j + 1u);
    double r = sqrt(-2.0 * log(u1));
    double ph = 6.283185307179586476925 * u2;
    return (m & 1u) ? r * sin(ph) : r * cos(ph);
}

/* ------------------------------------------------------- leaf generator */
typedef struct {
    int32_t kind;            /* 0 = uniform box, 1 = street-grid city */
    int32_t sh_degree;       /* 0..3 */
    double box[6];           /* kind 0: xmin xmax ymin ymax zmin zmax */
    double logscale_mu, logscale_sigma;
    double opacity_sigma;    /* opacity = sigmoid(N(0, sigma)) */
    double dc_sigma, band_sigma;
    /* kind 1 (city) */
    double city_extent;      /* square [0, extent]^2 */
    double street_spacing;   /* streets at k*spacing, k = 0..n_streets-1 */
    int32_t n_streets;
    double street_halfwidth; /* lateral offset U[-hw, hw] */
    double street_height;    /* height U[0, h] */
    double street_frac;      /* fraction of leaves on streets */
    double ground_sigma;     /* ground z = |N(0, sigma)| */
} sg_params;

static float sg_round_up_f32(double x) {
    float f = (float)x;
    if ((double)f < x) f = nextafterf(f, INFINITY);
    return f;
}

static float sg_round_down_f32(double x) {
    float f = (float)x;
    if ((double)f > x) f = nextafterf(f, -INFINITY);
    return f;
}

/*
 * Draw n leaf Gaussians.  Outputs (caller-allocated):
 *   mean[3n], cov6[6n] (xx xy xz yy yz zz), opacity[n],
 *   sh[n * 3 * (deg+1)^2] (coefficient-major, RGB innermost), rad2[n].
 */
int sg_gen_leaves(const sg_params* p, uint64_t n, uint64_t seed, float* mean,
                  float* cov6, float* opacity, float* sh, float* rad2) {
    if (!p || p->sh_degree < 0 || p->sh_degree > 3) return 1;
    const uint64_t key = sg_mix64(seed ^ 0x5EED5EED5EED5EEDull);
    const int K = (p->sh_degree + 1) * (p->sh_degree + 1);
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)n; ++i) {
        double m[3];
        if (p->kind == 0) {
            for (int a = 0; a < 3; ++a)
                m[a] = p->box[2 * a] + (p->box[2 * a + 1] - p->box[2 * a]) * sg_unif(key, i, a);
        } else {
            double L = p->city_extent;
            if (sg_unif(key, i, 3) < p->street_frac) {
                int along_x = sg_unif(key, i, 4) < 0.5;
                int k = (int)(sg_unif(key, i, 5) * p->n_streets);
                if (k >= p->n_streets) k = p->n_streets - 1;
                double line = k * p->street_spacing;
                double along = L * sg_unif(key, i, 6);
                double lat = p->street_halfwidth * (2.0 * sg_unif(key, i, 7) - 1.0);
                double h = p->street_height * sg_unif(key, i, 8);
                if (along_x) { m[0] = along; m[1] = line + lat; }
                else { m[0] = line + lat; m[1] = along; }
                m[2] = h;
            } else {
                m[0] = L * sg_unif(key, i, 9);
                m[1] = L * sg_unif(key, i, 10);
                m[2] = fabs(p->ground_sigma * sg_normal(key, i, 40));
            }
        }
        double s[3], q[4];
        for (int a = 0; a < 3; ++a)
            s[a] = exp(p->logscale_mu + p->logscale_sigma * sg_normal(key, i, (uint32_t)a));
        double qn = 0.0;
        for (int a = 0; a < 4; ++a) { q[a] = sg_normal(key, i, 4u + (uint32_t)a); qn += q[a] * q[a]; }
        qn = sqrt(qn);
        if (qn == 0.0) { q[0] = 1.0; q[1] = q[2] = q[3] = 0.0; qn = 1.0; }
        for (int a = 0; a < 4; ++a) q[a] /= qn;
        double w = q[0], x = q[1], y = q[2], z = q[3];
        double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z),     2 * (x * z + w * y),
                       2 * (x * y + w * z),     1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                       2 * (x * z - w * y),     2 * (y * z + w * x),     1 - 2 * (x * x + y * y)};
        double S[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += R[3 * r + k] * s[k] * s[k] * R[3 * c + k];
                S[3 * r + c] = acc;
            }
        for (int a = 0; a < 3; ++a) mean[3 * i + a] = (float)m[a];
        cov6[6 * i + 0] = (float)S[0]; cov6[6 * i + 1] = (float)S[1]; cov6[6 * i + 2] = (float)S[2];
        cov6[6 * i + 3] = (float)S[4]; cov6[6 * i + 4] = (float)S[5]; cov6[6 * i + 5] = (float)S[8];
        double on = p->opacity_sigma * sg_normal(key, i, 8u);
        opacity[i] = (float)(1.0 / (1.0 + exp(-on)));
        for (int k = 0; k < K; ++k)
            for (int c = 0; c < 3; ++c) {
                double sig = (k == 0) ? p->dc_sigma : p->band_sigma;
                sh[((size_t)i * K + k) * 3 + c] = (float)(sig * sg_normal(key, i, 10u + 3u * (uint32_t)k + (uint32_t)c));
            }
        double smax = s[0] > s[1] ? s[0] : s[1];
        smax = smax > s[2] ? smax : s[2];
        double R0 = 3.0 * smax;
        rad2[i] = sg_round_up_f32(R0 * R0);
    }
    return 0;
}

/* ------------------------------------------------------------ octree */
typedef struct {
    uint32_t lo, hi;      /* range into the Morton-sorted leaf order */
    int32_t lvl;          /* Morton level still to split; -1 = identical codes */
    uint32_t parent, first_child;
    uint32_t nchild, depth;
} sg_node;

typedef struct sg_tree {
    uint64_t n_leaves;
    uint64_t n_nodes;
    uint32_t max_depth;
    uint32_t* order;      /* Morton-sorted leaf indices */
    uint64_t* code;       /* codes in sorted order */
    sg_node* nodes;
    uint64_t* level_start; /* BFS level boundaries, max_depth + 2 entries */
} sg_tree;

static inline uint64_t sg_spread3(uint64_t v) { /* 21 bits -> every third bit */
    v &= 0x1FFFFFull;
    v = (v | (v << 32)) & 0x1F00000000FFFFull;
    v = (v | (v << 16)) & 0x1F0000FF0000FFull;
    v = (v | (v << 8)) & 0x100F00F00F00F00Full;
    v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

static inline uint32_t sg_digit(uint64_t code, int lvl) { return (uint32_t)((code >> (3 * lvl)) & 7u); }

/* first index in [lo, hi) whose digit at lvl is >= d (digits sorted there) */
static uint32_t sg_lower(const uint64_t* code, uint32_t lo, uint32_t hi, int lvl, uint32_t d) {
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (sg_digit(code[mid], lvl) < d) lo = mid + 1; else hi = mid;
    }
    return lo;
}

void sg_tree_free(sg_tree* t) {
    if (!t) return;
    free(t->order); free(t->code); free(t->nodes); free(t->level_start); free(t);
}

/* Build the topology over the leaf means.  Returns NULL on failure. */
sg_tree* sg_tree_build(uint64_t n, const float* mean) {
    if (n == 0 || n > 0x7FFFFFFFull) return NULL;
    sg_tree* t = (sg_tree*)calloc(1, sizeof(sg_tree));
    if (!t) return NULL;
    t->n_leaves = n;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            double v = mean[3 * i + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) if (hi[a] - lo[a] > ext) ext = hi[a] - lo[a];
    if (!(ext > 0.0)) ext = 1.0;
    const double scale = 2097152.0 / ext; /* 2^21 cells over the cube side */

    uint64_t* keys = (uint64_t*)malloc(n * sizeof(uint64_t));
    uint64_t* tmp = (uint64_t*)malloc(n * sizeof(uint64_t));
    uint32_t* ord = (uint32_t*)malloc(n * sizeof(uint32_t));
    uint32_t* ordt = (uint32_t*)malloc(n * sizeof(uint32_t));
    if (!keys || !tmp || !ord || !ordt) { free(keys); free(tmp); free(ord); free(ordt); sg_tree_free(t); return NULL; }
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)n; ++i) {
        uint64_t c = 0;
        for (int a = 0; a < 3; ++a) {
            double q = floor((mean[3 * i + a] - lo[a]) * scale);
            if (q < 0.0) q = 0.0;
            if (q > 2097151.0) q = 2097151.0;
            c |= sg_spread3((uint64_t)q) << (2 - a);
        }
        keys[i] = c;
        ord[i] = (uint32_t)i;
    }
    /* stable LSD radix sort of (code, index): 8 passes of 8 bits */
    size_t cnt[256];
    for (int pass = 0; pass < 8; ++pass) {
        int sh = pass * 8;
        memset(cnt, 0, sizeof(cnt));
        for (uint64_t k = 0; k < n; ++k) cnt[(keys[k] >> sh) & 255u]++;
        size_t run = 0;
        for (int d = 0; d < 256; ++d) { size_t c = cnt[d]; cnt[d] = run; run += c; }
        for (uint64_t k = 0; k < n; ++k) {
            size_t dst = cnt[(keys[k] >> sh) & 255u]++;
            tmp[dst] = keys[k];
            ordt[dst] = ord[k];
        }
        uint64_t* sw = keys; keys = tmp; tmp = sw;
        uint32_t* so = ord; ord = ordt; ordt = so;
    }
    free(tmp); free(ordt);
    t->order = ord;
    t->code = keys;

    size_t cap = 2 * (size_t)n;
    sg_node* nd = (sg_node*)malloc(cap * sizeof(sg_node));
    if (!nd) { sg_tree_free(t); return NULL; }
    nd[0].lo = 0; nd[0].hi = (uint32_t)n; nd[0].lvl = 20; nd[0].parent = 0xFFFFFFFFu;
    nd[0].first_child = 0; nd[0].nchild = 0; nd[0].depth = 0;
    size_t count = 1;
    uint32_t maxd = 0;
    /* breadth-first: node ids are queue positions */
    for (size_t q = 0; q < count; ++q) {
        sg_node cur = nd[q];
        if (cur.depth > maxd) maxd = cur.depth;
        if (cur.hi - cur.lo < 2) continue; /* leaf */
        uint32_t bounds[9];
        uint32_t nb = 0;
        int child_lvl = -1;
        int split = -1;
        if (cur.lvl >= 0) {
            for (int l = cur.lvl; l >= 0; --l)
                if (sg_digit(keys[cur.lo], l) != sg_digit(keys[cur.hi - 1], l)) { split = l; break; }
        }
        if (split >= 0) {
            bounds[nb++] = cur.lo;
            for (uint32_t d = 1; d < 8; ++d) {
                uint32_t b = sg_lower(keys, cur.lo, cur.hi, split, d);
                if (b > bounds[nb - 1] && b < cur.hi) bounds[nb++] = b;
            }
            bounds[nb++] = cur.hi;
            child_lvl = split - 1;
        } else {
            /* identical codes: up to 8 contiguous chunks of near-equal size */
            uint32_t len = cur.hi - cur.lo;
            uint32_t parts = len < 8 ? len : 8;
            for (uint32_t k = 0; k <= parts; ++k) bounds[nb++] = cur.lo + (uint32_t)(((uint64_t)len * k) / parts);
            child_lvl = -1;
        }
        uint32_t nch = nb - 1;
        if (count + nch > cap) { free(nd); sg_tree_free(t); return NULL; }
        nd[q].first_child = (uint32_t)count;
        nd[q].nchild = nch;
        for (uint32_t k = 0; k < nch; ++k) {
            sg_node c;
            c.lo = bounds[k]; c.hi = bounds[k + 1]; c.lvl = child_lvl;
            c.parent = (uint32_t)q; c.first_child = 0; c.nchild = 0; c.depth = cur.depth + 1;
            nd[count++] = c;
        }
    }
    t->nodes = nd;
    t->n_nodes = count;
    t->max_depth = maxd;
    t->level_start = (uint64_t*)calloc(maxd + 2, sizeof(uint64_t));
    if (!t->level_start) { sg_tree_free(t); return NULL; }
    /* BFS order => levels are contiguous */
    uint32_t lv = 0;
    t->level_start[0] = 0;
    for (size_t q = 0; q < count; ++q)
        while (nd[q].depth > lv) t->level_start[++lv] = q;
    t->level_start[maxd + 1] = count;
    return t;
}

uint64_t sg_tree_nodes(const sg_tree* t) { return t ? t->n_nodes : 0; }
uint32_t sg_tree_depth(const sg_tree* t) { return t ? t->max_depth : 0; }

/*
 * Fill the node arrays (caller-allocated, n_nodes entries each) from the
 * leaf attributes.  sh_dim = 3 * (deg+1)^2 floats per Gaussian.
 */
int sg_tree_fill(const sg_tree* t, int sh_dim, const float* lmean, const float* lcov6,
                 const float* lopac, const float* lsh, const float* lrad2, uint32_t* parent,
                 uint32_t* first_child, uint8_t* n_child, float* mean, float* cov6, float* opacity,
                 float* sh, float* radius2) {
    if (!t || sh_dim <= 0) return 1;
    const sg_node* nd = t->nodes;
    int64_t q;
    for (int64_t lv = (int64_t)t->max_depth; lv >= 0; --lv) {
        int64_t a = (int64_t)t->level_start[lv], b = (int64_t)t->level_start[lv + 1];
#pragma omp parallel for schedule(dynamic, 1024)
        for (q = a; q < b; ++q) {
            const sg_node* c = &nd[q];
            parent[q] = c->parent;
            first_child[q] = c->nchild ? c->first_child : 0u;
            n_child[q] = (uint8_t)c->nchild;
            if (c->nchild == 0) {
                uint32_t L = t->order[c->lo];
                for (int k = 0; k < 3; ++k) mean[3 * q + k] = lmean[3 * (size_t)L + k];
                for (int k = 0; k < 6; ++k) cov6[6 * q + k] = lcov6[6 * (size_t)L + k];
                opacity[q] = lopac[L];
                memcpy(&sh[(size_t)q * sh_dim], &lsh[(size_t)L * sh_dim], sizeof(float) * (size_t)sh_dim);
                radius2[q] = lrad2[L];
                continue;
            }
            uint32_t f0 = c->first_child, nc = c->nchild;
            double W = 0.0, prod = 1.0;
            for (uint32_t k = 0; k < nc; ++k) {
                double w = opacity[f0 + k];
                W += w;
                prod *= 1.0 - w;
            }
            int uniform = !(W > 0.0);
            if (uniform) W = (double)nc;
            double mu[3] = {0, 0, 0};
            for (uint32_t k = 0; k < nc; ++k) {
                double w = uniform ? 1.0 : (double)opacity[f0 + k];
                for (int a = 0; a < 3; ++a) mu[a] += w * (double)mean[3 * (size_t)(f0 + k) + a];
            }
            for (int a = 0; a < 3; ++a) mu[a] /= W;
            double S[6] = {0, 0, 0, 0, 0, 0};
            for (uint32_t k = 0; k < nc; ++k) {
                size_t ch = f0 + k;
                double w = uniform ? 1.0 : (double)opacity[ch];
                double d0 = mean[3 * ch] - mu[0], d1 = mean[3 * ch + 1] - mu[1], d2 = mean[3 * ch + 2] - mu[2];
                S[0] += w * (cov6[6 * ch + 0] + d0 * d0);
                S[1] += w * (cov6[6 * ch + 1] + d0 * d1);
                S[2] += w * (cov6[6 * ch + 2] + d0 * d2);
                S[3] += w * (cov6[6 * ch + 3] + d1 * d1);
                S[4] += w * (cov6[6 * ch + 4] + d1 * d2);
                S[5] += w * (cov6[6 * ch + 5] + d2 * d2);
            }
            for (int a = 0; a < 3; ++a) mean[3 * q + a] = (float)mu[a];
            for (int a = 0; a < 6; ++a) cov6[6 * q + a] = (float)(S[a] / W);
            for (int j = 0; j < sh_dim; ++j) {
                double acc = 0.0;
                for (uint32_t k = 0; k < nc; ++k) {
                    double w = uniform ? 1.0 : (double)opacity[f0 + k];
                    acc += w * (double)sh[(size_t)(f0 + k) * sh_dim + j];
                }
                sh[(size_t)q * sh_dim + j] = (float)(acc / W);
            }
            double op = uniform ? 0.0 : 1.0 - prod;
            if (op > 0.99) op = 0.99;
            opacity[q] = (float)op;
            /* nesting radius from the stored FP32 values */
            double R = 0.0;
            for (uint32_t k = 0; k < nc; ++k) {
                size_t ch = f0 + k;
                double d0 = (double)mean[3 * ch] - (double)mean[3 * q];
                double d1 = (double)mean[3 * ch + 1] - (double)mean[3 * q + 1];
                double d2 = (double)mean[3 * ch + 2] - (double)mean[3 * q + 2];
                double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2) + sqrt((double)radius2[ch]);
                if (r > R) R = r;
            }
            R *= 1.0 + 0x1p-12;
            radius2[q] = sg_round_up_f32(R * R);
        }
    }
    return 0;
}

/*
 * Nested axis-aligned node boxes, box[6 n ..] = lo x, y, z, hi x, y, z.
 * Children have larger ids than their parent, so one pass over descending
 * ids sees every child box before its parent's.
 */
int sg_tree_boxes(uint64_t n_nodes, const uint32_t* first_child, const uint8_t* n_child, const float* mean,
                  const float* cov6, float* box) {
    static const int diag[3] = {0, 3, 5};
    for (int64_t q = (int64_t)n_nodes - 1; q >= 0; --q) {
        float* b = box + 6 * (size_t)q;
        for (int a = 0; a < 3; ++a) {
            double v = (double)cov6[6 * (size_t)q + diag[a]];
            double h = 3.34 * sqrt(v > 0.0 ? v : 0.0);
            double m = (double)mean[3 * (size_t)q + a];
            b[a] = sg_round_down_f32(m - h);
            b[3 + a] = sg_round_up_f32(m + h);
        }
        for (uint32_t k = 0; k < n_child[q]; ++k) {
            const float* c = box + 6 * (size_t)(first_child[q] + k);
            for (int a = 0; a < 3; ++a) {
                if (c[a] < b[a]) b[a] = c[a];
                if (c[3 + a] > b[3 + a]) b[3 + a] = c[3 + a];
            }
        }
    }
    return 0;
}

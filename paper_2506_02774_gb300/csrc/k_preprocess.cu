// k_preprocess.cu -- culling & projection of the cut (paper Sec. 3.1
// 'Culling & Projection') with the preemptive alpha filter moved into it
// (Sec. 4.2, Eq. 4: alpha >= alpha* <=> rho >= ln alpha* - ln theta).
//
// One thread per cut node in front of the near plane (the LoD stage lists
// them, in ascending node id), dense and barrier-free: every entry's record
// is written at its own index, and a culled entry gets the depth key
// 0xFFFFFFFF.  The stable depth sort then puts the visible Gaussians first,
// ordered by (depth key, node id), with no compaction pass at all.
//
// Per node: p = R (mu - C); depth key = FP32 bits of
// ((R20 dx + R21 dy) + R22 dz) with single-rounded operations; culled when
// z <= z_near.  Gaussian-level filter: theta < alpha* is dropped.  EWA:
// Sigma' = M Sigma M^T + 0.3 I with M = J R, J the perspective Jacobian with
// x/z, y/z clamped to 1.3 (W/2)/fx, 1.3 (H/2)/fy.  Footprint box from
// r^2 = 2 (ln theta - ln alpha*) (plus the 2e-3 test slack); candidate tiles
// are those whose pixel-centre rectangle meets the box.  A Gaussian is kept
// when it has at least one candidate tile; the tile-level test (Eq. 4 over
// each candidate tile) runs in the emission, where the work is balanced over
// candidate slots.  Colour (real SH up to degree 3, +0.5, clamped at 0) is
// evaluated here too, for the visible entries: the SH row (192 bytes in FP32
// at degree 3) is requested together with the centre and the covariance, so
// the projection arithmetic runs while it arrives, and the kernel streams
// all of a node's bytes in one pass (two 256-thread CTAs per SM, registers
// for the whole row in flight).  As a separate pass the colour could not
// overlap the latency-bound sorts, which hold every SM slot they can get.
#include <cuda_fp16.h>

#include "vgr_internal.cuh"
#include "vgr_launch.h"

namespace vgr {

constexpr int PRE_THREADS = 256;

// Real spherical harmonics (orthonormal, Condon-Shortley phase) as
// polynomials of the unit direction; constants are the closed forms
//  l=0: 1/(2 sqrt(pi))
//  l=1: sqrt(3/(4 pi))
//  l=2: sqrt(15/(4 pi)), sqrt(5/(16 pi)), sqrt(15/(16 pi))
//  l=3: sqrt(35/(32 pi)), sqrt(105/(4 pi)), sqrt(21/(32 pi)), sqrt(7/(16 pi)), sqrt(105/(16 pi))
template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
    Y[0] = 0.28209479177387814f;
    if (DEG >= 1) {
        Y[1] = -0.48860251190291992f * y;
        Y[2] = 0.48860251190291992f * z;
        Y[3] = -0.48860251190291992f * x;
    }
    if (DEG >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = 1.0925484305920792f * (x * y);
        Y[5] = -1.0925484305920792f * (y * z);
        Y[6] = 0.31539156525252005f * (2.0f * zz - xx - yy);
        Y[7] = -1.0925484305920792f * (x * z);
        Y[8] = 0.54627421529603959f * (xx - yy);
        if (DEG >= 3) {
            Y[9] = -0.59004358992664352f * y * (3.0f * xx - yy);
            Y[10] = 2.8906114426405538f * (x * y) * z;
            Y[11] = -0.45704579946446572f * y * (4.0f * zz - xx - yy);
            Y[12] = 0.37317633259011540f * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
            Y[13] = -0.45704579946446572f * x * (4.0f * zz - xx - yy);
            Y[14] = 1.4453057213202769f * z * (xx - yy);
            Y[15] = -0.59004358992664352f * x * (xx - 3.0f * yy);
        }
    }
}

template <int STORE>
struct Store;

template <>
struct Store<VGR_STORE_FP32> {
    __device__ static __forceinline__ void cov(const SceneDev& sc, uint32_t n, float* S, float& theta, float& lnth) {
        const float4 a = sc.covA[n], b = sc.covB[n];
        S[0] = a.x; S[1] = a.y; S[2] = a.z; S[3] = a.w; S[4] = b.x; S[5] = b.y;
        theta = b.z;
        lnth = b.w;
    }
    template <int K>
    __device__ static __forceinline__ void sh(const SceneDev& sc, uint32_t n, float* c) {
        const float4* p = reinterpret_cast<const float4*>(sc.sh) + (size_t)n * (sc.sh_stride / 4);
        constexpr int NV = (3 * K + 3) / 4;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const float4 v = __ldg(p + i);
            c[4 * i + 0] = v.x; c[4 * i + 1] = v.y; c[4 * i + 2] = v.z; c[4 * i + 3] = v.w;
        }
    }
};

template <>
struct Store<VGR_STORE_HALF> {
    // covariance as 6 BF16 in covA (uint4 storage: xx xy xz yy yz zz, 2 spare),
    // opacity and ln(opacity) FP32 in covB.xy
    __device__ static __forceinline__ void cov(const SceneDev& sc, uint32_t n, float* S, float& theta, float& lnth) {
        const uint4 a = reinterpret_cast<const uint4*>(sc.covA)[n];
        const float4 b = sc.covB[n];
        const uint32_t w[3] = {a.x, a.y, a.z};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            S[2 * i] = __uint_as_float(w[i] << 16);
            S[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
        }
        theta = b.x;
        lnth = b.y;
    }
    template <int K>
    __device__ static __forceinline__ void sh(const SceneDev& sc, uint32_t n, float* c) {
        const uint4* p = reinterpret_cast<const uint4*>(sc.sh) + (size_t)n * (sc.sh_stride / 8);
        constexpr int NV = (3 * K + 7) / 8;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const uint4 v = __ldg(p + i);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const __half2 h = *reinterpret_cast<const __half2*>(&w[j]);
                const float2 f = __half22float2(h);
                c[8 * i + 2 * j] = f.x;
                c[8 * i + 2 * j + 1] = f.y;
            }
        }
    }
};

template <int DEG, int STORE, bool INTERP>
__global__ void __launch_bounds__(PRE_THREADS, 2) k_preprocess(SceneDev sc, const uint32_t* __restrict__ front,
                                                            const uint32_t* __restrict__ n_front_p, uint32_t cap,
                                                            const FrameParams* __restrict__ fp, VisBuffers vis,
                                                            Counters* __restrict__ ctr) {
    pdl_wait();
    constexpr int K = (DEG + 1) * (DEG + 1);  // SH coefficients per channel
    constexpr int NSH = ((3 * K + 7) / 8) * 8;
    __shared__ uint32_t s_hist[4][256];  // digit histograms of the depth keys (the sort's passes)
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) (&s_hist[0][0])[i] = 0u;
    __syncthreads();
    const uint32_t n_front = min(*n_front_p, cap);
    const float R0 = fp->R[0], R1 = fp->R[1], R2 = fp->R[2], R3 = fp->R[3], R4 = fp->R[4], R5 = fp->R[5];
    const float R6 = fp->R[6], R7 = fp->R[7], R8 = fp->R[8];
    const float Cx = fp->pos[0], Cy = fp->pos[1], Cz = fp->pos[2];
    const float fx = fp->fx, fy = fp->fy, cx = fp->cx, cy = fp->cy, z_near = fp->z_near;
    const float limx = fp->limx, limy = fp->limy, Wf = fp->width_f, Hf = fp->height_f;
    const int TW = (int)fp->tiles_x, TH = (int)fp->tiles_y;
    const float Tf = (float)fp->tile, iT = 1.0f / Tf;  // tile side (a power of two: exact)
    const bool canonical = fp->filter == VGR_FILTER_CANONICAL;
    const float lod_t = fp->lod_t;
    uint32_t n_visible = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    // uniform trip count per warp so the visible count can use a ballot
    // the next round's node id is loaded one round ahead
    const uint32_t first = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u;
    uint32_t node_next = first + lane_id() < n_front ? front[first + lane_id()] : 0u;
    for (uint32_t base = first; base < n_front; base += stride) {
        const uint32_t i = base + lane_id();
        bool v = i < n_front;
        uint32_t node = node_next, zbits = 0xFFFFFFFFu;
        node_next = i + stride < n_front ? front[i + stride] : 0u;
        float u = 0.f, vv = 0.f, ca = 0.f, cb = 0.f, cc = 0.f, thr = 0.f, theta = 0.f, lw = 0.f;
        uint32_t box_hw = 0u;  // footprint box half-height | half-width << 16, FP16 rounded up
        int tx0 = 0, ty0 = 0, tx1 = -1, ty1 = -1;
        if (v) {
            float4 m = sc.cr[node];
            float shc[NSH];
            Store<STORE>::template sh<K>(sc, node, shc);  // in flight with the centre and covariance
            float S[6], lnth = 0.f;
            Store<STORE>::cov(sc, node, S, theta, lnth);  // in flight together with the centre
            if constexpr (INTERP) {
                // the rendered Gaussian moves towards the parent's by the weight w:
                // mean (single-rounded), covariance and opacity; the parent's
                // opacity is shared among its k children, 1 - (1 - theta_p)^(1/k),
                // so that k coincident copies have the parent's peak opacity
                const uint32_t p = sc.parent[node];
                if (p != NONE) {
                    const float4 mp = sc.cr[p];
                    lw = lod_interp_weight(lod_size_ratio(m, Cx, Cy, Cz), lod_size_ratio(mp, Cx, Cy, Cz), lod_t);
                    if (lw > 0.f) {
                        float Sp[6], thp, lnp;
                        Store<STORE>::cov(sc, p, Sp, thp, lnp);
                        const float kp = (float)(sc.child[p] >> CHILD_SHIFT);
                        m.x = lod_lerp_rn(m.x, mp.x, lw);
                        m.y = lod_lerp_rn(m.y, mp.y, lw);
                        m.z = lod_lerp_rn(m.z, mp.z, lw);
#pragma unroll
                        for (int j = 0; j < 6; ++j) S[j] = fmaf(lw, Sp[j] - S[j], S[j]);
                        const float share = -expm1f(log1pf(-thp) / kp);
                        theta = fmaf(lw, share - theta, theta);
                        lnth = logf(theta);
                    }
                }
            }
            const float dx = __fsub_rn(m.x, Cx), dy = __fsub_rn(m.y, Cy), dz = __fsub_rn(m.z, Cz);
            const float z = __fadd_rn(__fadd_rn(__fmul_rn(R6, dx), __fmul_rn(R7, dy)), __fmul_rn(R8, dz));
            v = z > z_near;  // always true for the in-front list; kept as the definition
            if (v && !canonical && !(theta >= ALPHA_MIN)) v = false;  // Gaussian-level filter
            if (v) {
                const float x = fmaf(R0, dx, fmaf(R1, dy, R2 * dz));
                const float y = fmaf(R3, dx, fmaf(R4, dy, R5 * dz));
                const float iz = 1.0f / z;
                const float xz = x * iz, yz = y * iz;
                u = fmaf(fx, xz, cx);
                vv = fmaf(fy, yz, cy);
                const float tx = fminf(limx, fmaxf(-limx, xz));
                const float ty = fminf(limy, fmaxf(-limy, yz));
                const float fxz = fx * iz, fyz = fy * iz;
                // M = J R: rows M0 = fx/z (R0row - tx R2row), M1 = fy/z (R1row - ty R2row)
                const float m00 = fxz * fmaf(-tx, R6, R0), m01 = fxz * fmaf(-tx, R7, R1), m02 = fxz * fmaf(-tx, R8, R2);
                const float m10 = fyz * fmaf(-ty, R6, R3), m11 = fyz * fmaf(-ty, R7, R4), m12 = fyz * fmaf(-ty, R8, R5);
                // Sigma M0^T, Sigma M1^T (Sigma = [[S0 S1 S2] [S1 S3 S4] [S2 S4 S5]])
                const float a0 = fmaf(S[0], m00, fmaf(S[1], m01, S[2] * m02));
                const float a1 = fmaf(S[1], m00, fmaf(S[3], m01, S[4] * m02));
                const float a2 = fmaf(S[2], m00, fmaf(S[4], m01, S[5] * m02));
                const float b0 = fmaf(S[0], m10, fmaf(S[1], m11, S[2] * m12));
                const float b1 = fmaf(S[1], m10, fmaf(S[3], m11, S[4] * m12));
                const float b2 = fmaf(S[2], m10, fmaf(S[4], m11, S[5] * m12));
                const float s00 = fmaf(m00, a0, fmaf(m01, a1, m02 * a2)) + DILATE;
                const float s01 = fmaf(m10, a0, fmaf(m11, a1, m12 * a2));
                const float s11 = fmaf(m10, b0, fmaf(m11, b1, m12 * b2)) + DILATE;
                // det = s00 s11 - s01^2 with the product error recovered (Kahan)
                const float w = s01 * s01;
                const float e = fmaf(-s01, s01, w);
                const float det = fmaf(s00, s11, -w) + e;
                if (!(det > 0.f)) {
                    v = false;
                } else {
                    const float idet = 1.0f / det;
                    ca = s11 * idet;
                    cb = -s01 * idet;
                    cc = s00 * idet;
                    thr = LN_ALPHA_MIN - lnth;
                    float bx, by;
                    if (!canonical) {
                        // opacity-aware box of {rho >= thr - slack}
                        const float r2 = fmaxf(0.f, 2.0f * (lnth - LN_ALPHA_MIN) + 2.0f * TILE_EPS);
                        bx = sqrtf(r2 * s00) * 1.0001f + 1e-3f;
                        by = sqrtf(r2 * s11) * 1.0001f + 1e-3f;
                    } else {
                        // 3-sigma radius of the larger eigenvalue (3DGS-style square footprint)
                        const float mid = 0.5f * (s00 + s11);
                        const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
                        bx = by = ceilf(3.0f * sqrtf(lam));
                    }
                    tx0 = max(0, (int)ceilf((u - bx - (Tf - 0.5f)) * iT));
                    tx1 = min(TW - 1, (int)floorf((u + bx - 0.5f) * iT));
                    ty0 = max(0, (int)ceilf((vv - by - (Tf - 0.5f)) * iT));
                    ty1 = min(TH - 1, (int)floorf((vv + by - 0.5f) * iT));
                    if (!(u - bx < Wf + Tf) || !(u + bx > -Tf) || !(vv - by < Hf + Tf) || !(vv + by > -Tf)) {
                        tx1 = -1;  // far outside (also guards the float->int conversions)
                    }
                    if (tx0 > tx1 || ty0 > ty1) v = false;
                    box_hw = (uint32_t)__half_as_ushort(__float2half_ru(by)) |
                             ((uint32_t)__half_as_ushort(__float2half_ru(bx)) << 16);
                }
            }
            if (v) {
                // colour: rgb = sum_lm c_lm Y_lm(d) + 0.5, clamped at 0, d = (mu - C)/|mu - C|
                // (with interpolation the coefficients and the mean move towards the parent's)
                if constexpr (INTERP) {
                    if (lw > 0.f) {
                        float shp[NSH];
                        Store<STORE>::template sh<K>(sc, sc.parent[node], shp);
#pragma unroll
                        for (int j = 0; j < 3 * K; ++j) shc[j] = fmaf(lw, shp[j] - shc[j], shc[j]);
                    }
                }
                float Y[K];
                const float inv = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                sh_basis<DEG>(dx * inv, dy * inv, dz * inv, Y);
                float cr = 0.5f, cg = 0.5f, cbl = 0.5f;
#pragma unroll
                for (int kk = 0; kk < K; ++kk) {
                    cr = fmaf(shc[3 * kk + 0], Y[kk], cr);
                    cg = fmaf(shc[3 * kk + 1], Y[kk], cg);
                    cbl = fmaf(shc[3 * kk + 2], Y[kk], cbl);
                }
                vis.rgb[i] = make_float4(fmaxf(cr, 0.f), fmaxf(cg, 0.f), fmaxf(cbl, 0.f), 0.f);
                zbits = __float_as_uint(z);
            }
        }
        n_visible += __popc(__ballot_sync(0xFFFFFFFFu, v));
        // one shared-memory atomic per digit: equal digits within the warp (the
        // high bytes of neighbouring nodes' depths) are combined by the hardware,
        // cheaper than finding the peers first
        if (i < n_front) {
#pragma unroll
            for (int p = 0; p < 4; ++p) atomicAdd(&s_hist[p][(zbits >> (8 * p)) & 255u], 1u);
        }
        if (i < n_front) {
            vis.depth[i] = zbits;  // culled: all ones, sorted behind every visible key
            vis.ntile[i] = v ? (uint32_t)(tx1 - tx0 + 1) * (uint32_t)(ty1 - ty0 + 1) : 0u;
            vis.rect[i] = make_uint2((uint32_t)tx0 | ((uint32_t)ty0 << 16), (uint32_t)tx1 | ((uint32_t)ty1 << 16));
            vis.recA[i] = make_float4(u, vv, -0.5f * ca, -cb);
            vis.recB[i] = make_float4(-0.5f * cc, thr, theta, __uint_as_float(box_hw));
            if (INTERP) vis.lw[i] = lw;
        }
    }
    if (lane_id() == 0 && n_visible) atomicAdd(&ctr->n_vis, n_visible);
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) {
        const uint32_t c = (&s_hist[0][0])[i];
        if (c) atomicAdd(&ctr->depth_hist[0][0] + i, c);
    }
}

// ln(opacity) next to the opacity (Eq. 4 needs ln theta per Gaussian)
__global__ void k_prepare(float4* covB, uint32_t n, int half) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float4 b = covB[i];
        if (half) b.y = logf(b.x);
        else b.w = logf(b.z);
        covB[i] = b;
    }
}

void prepare_scene(float4* covB, uint32_t n, cudaStream_t s) {
    k_prepare<<<1024, 256, 0, s>>>(covB, n, 0);
}
void prepare_scene_half(float4* covB, uint32_t n, cudaStream_t s) {
    k_prepare<<<1024, 256, 0, s>>>(covB, n, 1);
}

void launch_preprocess(const SceneDev& sc, const uint32_t* front, const uint32_t* n_front, uint32_t cap,
                       const FrameParams* fp, VisBuffers vis, Counters* ctr, bool interp, int grid, cudaStream_t s) {
    const bool half = sc.storage == VGR_STORE_HALF;
#define VGR_PRE_LAUNCH(D, ST, IN) \
    launch_k(k_preprocess<D, ST, IN>, grid, PRE_THREADS, s, sc, front, n_front, cap, fp, vis, ctr)
#define VGR_PRE_CASE(D)                                            \
    case D:                                                        \
        if (interp) {                                              \
            if (half) VGR_PRE_LAUNCH(D, VGR_STORE_HALF, true);     \
            else VGR_PRE_LAUNCH(D, VGR_STORE_FP32, true);          \
        } else {                                                   \
            if (half) VGR_PRE_LAUNCH(D, VGR_STORE_HALF, false);    \
            else VGR_PRE_LAUNCH(D, VGR_STORE_FP32, false);         \
        }                                                          \
        break;
    switch (sc.sh_degree) {
        VGR_PRE_CASE(0)
        VGR_PRE_CASE(1)
        VGR_PRE_CASE(2)
        VGR_PRE_CASE(3)
        default: break;
    }
#undef VGR_PRE_CASE
#undef VGR_PRE_LAUNCH
}

uint32_t preprocess_tile() { return PRE_THREADS; }

}  // namespace vgr

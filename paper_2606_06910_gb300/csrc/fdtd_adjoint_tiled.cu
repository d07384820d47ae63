// TMA-tiled discrete adjoint step: the transpose of one forward step as two
// z-march kernels that mirror the forward stages (paper Sec. 3.1-3.2 taken in
// reverse; see fdtd_adjoint.cu for the assignment-by-assignment transpose):
//
//   stage A (adjoint of the pressure step), per node:
//     q = kdt lam_p                      (kdt = -dt K / vscale)
//     lam_h_d = q + [d-slab] ((kinv_d - 1) q + a_d (lam_psip_d + q))
//     lam_v_d -= D_d lam_h_d ; lam_psip_d <- b_d (lam_psip_d + q) ; dJ/dK += -(dt/vscale) S lam_p
//   stage B (adjoint of the velocity half step), per node:
//     r_d = -dtr lam_v_d
//     lam_g_d = r_d + [d-slab] ((kinv_d - 1) r_d + a_d (lam_psiv_d + r_d))
//     lam_p -= sum_d D_d lam_g_d ; lam_psiv_d <- b_d (lam_psiv_d + r_d)
//
// Each kernel stages one plane per iteration by TMA (the field it
// differentiates with a 4-node halo, zero-filled beyond the grid), forms
// lam_h / lam_g for x and y in shared memory, and keeps the z direction in a
// 9-plane register queue.  lam_p and lam_v are updated in place (each stage
// reads at its halo only the field it does not write); the memory variables
// are double-buffered.  FP32 only.
#include "fdtd_internal.cuh"

namespace fdtd {

constexpr int AHALO = 4;
constexpr int AW = TX + 2 * AHALO;    // 40: x extent with halo
constexpr int AHT = TY + 2 * AHALO;   // 40: y extent with halo
constexpr int ANS = 3;                // TMA stages

struct AdjTiledArgs {
    Geom g;
    int tiles_x, zchunk;
    const float *kdt;
    float *ap;
    float *av[3];
    const float *apsiv_in[3];
    float *apsiv_out[3];
    const float *apsip_in[3];
    float *apsip_out[3];
    const float *cb[3], *ca[3], *ck[3];
    float c[4];
    float dtr;
    float dt_over_vs;
    const float *s_tape;   // [nshots][vol] bracket of this step
    float *gradK;          // [nshots][vol]
    unsigned *err;
};

__device__ __forceinline__ F4 ld4s(const float *p)
{
    const float4 q = *reinterpret_cast<const float4 *>(p);
    return F4{{q.x, q.y, q.z, q.w}};
}
__device__ __forceinline__ void st4s(float *p, const F4 &v)
{
    *reinterpret_cast<float4 *>(p) = make_float4(v.v[0], v.v[1], v.v[2], v.v[3]);
}
__device__ __forceinline__ F4 f4z() { return F4{{0.f, 0.f, 0.f, 0.f}}; }

// D along a row: outputs at columns c0..c0+3 of `row` (c0 >= 4, multiple of 4)
__device__ __forceinline__ F4 drow(const float *row, int c0, const float *w)
{
    const F4 a = ld4s(row + c0 - 4), b = ld4s(row + c0), c = ld4s(row + c0 + 4);
    const float f[12] = {a.v[0], a.v[1], a.v[2], a.v[3], b.v[0], b.v[1], b.v[2], b.v[3], c.v[0], c.v[1], c.v[2], c.v[3]};
    F4 r;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        r.v[i] = w[0] * (f[i + 5] - f[i + 3]) + w[1] * (f[i + 6] - f[i + 2]) + w[2] * (f[i + 7] - f[i + 1]) +
                 w[3] * (f[i + 8] - f[i]);
    return r;
}

// D along a column: rows r0 +- l, 4 columns at c of a plane with `stride`
__device__ __forceinline__ F4 dcol(const float *plane, int stride, int r0, int c, const float *w)
{
    F4 r = f4z();
#pragma unroll
    for (int l = 1; l <= 4; ++l) {
        const F4 p = ld4s(plane + (r0 + l) * stride + c), m = ld4s(plane + (r0 - l) * stride + c);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            r.v[i] += w[l - 1] * (p.v[i] - m.v[i]);
    }
    return r;
}

__device__ __forceinline__ F4 dq(const F4 *q, const float *w)   // queue q[0..8], centre 4
{
    F4 r;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        r.v[i] = w[0] * (q[5].v[i] - q[3].v[i]) + w[1] * (q[6].v[i] - q[2].v[i]) + w[2] * (q[7].v[i] - q[1].v[i]) +
                 w[3] * (q[8].v[i] - q[0].v[i]);
    return r;
}

// lam <- lam + [slab] ((kinv - 1) lam + a (psi + lam)) for 4 nodes sharing a
// profile value (y or z slab)
__device__ __forceinline__ F4 corr_uniform(const F4 &lam, const F4 &psi, float a, float k)
{
    F4 r;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        r.v[i] = lam.v[i] + (k - 1.f) * lam.v[i] + a * (psi.v[i] + lam.v[i]);
    return r;
}

struct AdjSmemA {
    static constexpr int AP = 0;                  // [AHT][AW]
    static constexpr int KD = AP + AHT * AW;      // [AHT][AW]
    static constexpr int APQ = KD + AHT * AW;     // [TY][TX]
    static constexpr int KDQ = APQ + TY * TX;     // [TY][TX]
    static constexpr int STAGE = KDQ + TY * TX;   // floats per stage
    static constexpr int HX = ANS * STAGE;        // [TY][AW]
    static constexpr int HY = HX + TY * AW;       // [AHT][TX]
    static constexpr int CX = HY + AHT * TX;      // [3][AW] coefficients over the x range
    static constexpr int END = CX + 3 * AW;
    static constexpr int BYTES = END * 4 + 8 * ANS;
    static_assert((STAGE * 4) % 128 == 0 && (AP * 4) % 128 == 0 && (KD * 4) % 128 == 0 && (APQ * 4) % 128 == 0 &&
                      (KDQ * 4) % 128 == 0,
                  "TMA destinations must stay 128-byte aligned");
};

struct AdjSmemB {
    static constexpr int VX = 0;                  // [TY][AW]  lam_v_x with x halo
    static constexpr int VY = VX + TY * AW;       // [AHT][TX] lam_v_y with y halo
    static constexpr int VZQ = VY + AHT * TX;     // [TY][TX]  lam_v_z at t + 4
    static constexpr int STAGE = VZQ + TY * TX;
    static constexpr int GX = ANS * STAGE;        // [TY][AW]
    static constexpr int GY = GX + TY * AW;       // [AHT][TX]
    static constexpr int CX = GY + AHT * TX;      // [3][AW]
    static constexpr int END = CX + 3 * AW;
    static constexpr int BYTES = END * 4 + 8 * ANS;
    static_assert((STAGE * 4) % 128 == 0 && (VY * 4) % 128 == 0 && (VZQ * 4) % 128 == 0,
                  "TMA destinations must stay 128-byte aligned");
};

// per-tile CPML coefficients of the x range [x0-4, x0+TX+4): 0, 0, 1 outside the slab / grid
__device__ __forceinline__ void load_cx(float *cx, const AdjTiledArgs &A, int x0)
{
    const Geom &G = A.g;
    for (int i = threadIdx.x; i < 3 * AW; i += NTHREADS) {
        const int c = i / AW, x = x0 - AHALO + i % AW;
        const bool in = x >= 0 && x < G.nx && in_slab(x, G.nx, G.lo[0], G.hi[0]);
        cx[i] = in ? (c == 0 ? A.cb[0][x] : (c == 1 ? A.ca[0][x] : A.ck[0][x])) : (c == 2 ? 1.f : 0.f);
    }
}

// x-slab correction of 4 nodes starting at x (row y, plane z) in place, with
// the memory variable from psi (vector layout of the x slab), coefficients
// from the tile cache at column cc
__device__ __forceinline__ void corr_x(F4 &lam, const Geom &G, const float *psi, const float *cx, int cc, int z, int y,
                                       int x)
{
    if (x < 0 || x >= G.nx || y >= G.ny || !(x < G.lo[0] || x + 3 >= G.nx - G.hi[0]))
        return;
    const F4 ps = ld4s(psi + slab_index(G, 0, z, y, x));
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float a = cx[AW + cc + i], k = cx[2 * AW + cc + i];
        lam.v[i] = lam.v[i] + (k - 1.f) * lam.v[i] + a * (ps.v[i] + lam.v[i]);
    }
}

__global__ void __launch_bounds__(NTHREADS, 2)
    adj_tiled_a_kernel(const __grid_constant__ CUtensorMap mAP, const __grid_constant__ CUtensorMap mAPq,
                       const __grid_constant__ CUtensorMap mKD, const __grid_constant__ CUtensorMap mKDq,
                       const AdjTiledArgs A)
{
    using L = AdjSmemA;
    extern __shared__ __align__(1024) float sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L::END);
    const Geom &G = A.g;
    const int tid = threadIdx.x, tx = tid % (TX / 4), ty = tid / (TX / 4);
    const int tile = blockIdx.x;
    const int x0 = (tile % A.tiles_x) * TX, y0 = (tile / A.tiles_x) * TY;
    const int z0 = blockIdx.y * A.zchunk, z1 = min(G.nz, z0 + A.zchunk);
    const int shot = blockIdx.z;
    const int gx = x0 + 4 * tx, gy = y0 + ty;
    const bool row_ok = gy < G.ny && gx < G.nxp;
    const int niter = z1 - z0 + 8;
    const float w[4] = {A.c[0], A.c[1], A.c[2], A.c[3]};
    const long long fo = (long long)shot * G.vol;
    const int nv = G.nx - gx;   // lanes of this thread inside the grid (the row padding stays untouched)
    const float *psin[3];
    float *psout[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        psin[d] = A.apsip_in[d] + (long long)shot * G.slab[d];
        psout[d] = A.apsip_out[d] + (long long)shot * G.slab[d];
    }
    const bool xs_tile = G.w[0] > 0 && (x0 - AHALO < G.lo[0] || x0 + TX + AHALO > G.nx - G.hi[0]);
    const bool ys_tile = G.w[1] > 0 && (y0 - AHALO < G.lo[1] || y0 + TY + AHALO > G.ny - G.hi[1]);
    float *cx = sm + L::CX;
    load_cx(cx, A, x0);

    if (tid == 0) {
        prefetch_tmap(&mAP);
        prefetch_tmap(&mAPq);
        prefetch_tmap(&mKD);
        prefetch_tmap(&mKDq);
        for (int s = 0; s < ANS; ++s)
            mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int it) {
        const int t = z0 - 8 + it;
        float *S = sm + (it % ANS) * L::STAGE;
        uint64_t *b = &bar[it % ANS];
        const bool q_on = t + 4 >= 0 && t + 4 < G.nz, main_on = t >= z0;
        uint32_t bytes = (q_on ? 2u * TY * TX * 4u : 0u) + (main_on ? 2u * AHT * AW * 4u : 0u);
        mbar_arrive_expect_tx(b, bytes);
        if (q_on) {
            tma_load_4d(S + L::APQ, &mAPq, b, x0, y0, t + 4, shot);
            tma_load_3d(S + L::KDQ, &mKDq, b, x0, y0, t + 4);
        }
        if (main_on) {
            tma_load_4d(S + L::AP, &mAP, b, x0 - AHALO, y0 - AHALO, t, shot);
            tma_load_3d(S + L::KD, &mKD, b, x0 - AHALO, y0 - AHALO, t);
        }
    };
    if (tid == 0)
        for (int i = 0; i < ANS && i < niter; ++i)
            issue(i);

    F4 hq[9];   // lam_h_z(t - 4 + j)
#pragma unroll
    for (int j = 0; j < 9; ++j)
        hq[j] = f4z();

    for (int it = 0; it < niter; ++it) {
        const int t = z0 - 8 + it;
        const float *S = sm + (it % ANS) * L::STAGE;
        const bool ok = mbar_wait_bounded(&bar[it % ANS], (it / ANS) & 1, WAIT_LIMIT);

        // ---- lam_h_z at plane t + 4 into the queue
        F4 hn = f4z();
        const int zq = t + 4;
        if (ok && zq >= 0 && zq < G.nz) {
            const F4 a = ld4s(S + L::APQ + ty * TX + 4 * tx), k = ld4s(S + L::KDQ + ty * TX + 4 * tx);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                hn.v[i] = a.v[i] * k.v[i];
            if (row_ok && in_slab(zq, G.nz, G.lo[2], G.hi[2]))
                hn = corr_uniform(hn, ld4s(psin[2] + slab_index(G, 2, zq, gy, gx)), __ldg(A.ca[2] + zq),
                                  __ldg(A.ck[2] + zq));
        }
        hq[8] = hn;

        const bool active = t >= z0;
        if (ok && active) {
            // ---- lam_h_x (own rows, x halo) and lam_h_y (y halo, own columns)
            float *HX = sm + L::HX, *HY = sm + L::HY;
            for (int v = tid; v < TY * AW / 4; v += NTHREADS) {
                const int r = v / (AW / 4), c = 4 * (v % (AW / 4));
                const F4 a = ld4s(S + L::AP + (r + AHALO) * AW + c), k = ld4s(S + L::KD + (r + AHALO) * AW + c);
                F4 h;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    h.v[i] = a.v[i] * k.v[i];
                if (xs_tile)
                    corr_x(h, G, psin[0], cx, c, t, y0 + r, x0 - AHALO + c);
                st4s(HX + r * AW + c, h);
            }
            for (int v = tid; v < AHT * TX / 4; v += NTHREADS) {
                const int r = v / (TX / 4), c = 4 * (v % (TX / 4));
                const F4 a = ld4s(S + L::AP + r * AW + c + AHALO), k = ld4s(S + L::KD + r * AW + c + AHALO);
                F4 h;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    h.v[i] = a.v[i] * k.v[i];
                const int y = y0 - AHALO + r;
                if (ys_tile && y >= 0 && y < G.ny && x0 + c < G.nxp && in_slab(y, G.ny, G.lo[1], G.hi[1]))
                    h = corr_uniform(h, ld4s(psin[1] + slab_index(G, 1, t, y, x0 + c)), __ldg(A.ca[1] + y),
                                     __ldg(A.ck[1] + y));
                st4s(HY + r * TX + c, h);
            }
        }
        if (__syncthreads_or(ok ? 0 : 1)) {
            if (tid == 0) {
                atomicOr(A.err, ERR_TIMEOUT);
                for (int j = it; j < niter && j < it + ANS; ++j)
                    mbar_wait_bounded(&bar[j % ANS], (j / ANS) & 1, WAIT_LIMIT_DRAIN);
            }
            return;
        }
        if (active && row_ok) {
            const long long o = fo + (long long)t * G.plane + (long long)gy * G.nxp + gx;
            const F4 dvx = drow(sm + L::HX + ty * AW, 4 * tx + AHALO, w);
            const F4 dvy = dcol(sm + L::HY, TX, ty + AHALO, 4 * tx, w);
            const F4 dvz = dq(hq, w);
            F4 vx = ld4s(A.av[0] + o), vy = ld4s(A.av[1] + o), vz = ld4s(A.av[2] + o);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (i < nv) {
                    vx.v[i] -= dvx.v[i];
                    vy.v[i] -= dvy.v[i];
                    vz.v[i] -= dvz.v[i];
                }
            st4s(A.av[0] + o, vx);
            st4s(A.av[1] + o, vy);
            st4s(A.av[2] + o, vz);
            // own q = kdt lam_p, memory variables and dJ/dK
            const F4 apo = ld4s(S + L::AP + (ty + AHALO) * AW + 4 * tx + AHALO);
            const F4 kdo = ld4s(S + L::KD + (ty + AHALO) * AW + 4 * tx + AHALO);
            F4 q;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                q.v[i] = apo.v[i] * kdo.v[i];
            if (xs_tile && gy < G.ny && gx < G.nx && (gx < G.lo[0] || gx + 3 >= G.nx - G.hi[0])) {
                const long long si = slab_index(G, 0, t, gy, gx);
                const F4 ps = ld4s(psin[0] + si);
                F4 pn;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    pn.v[i] = cx[4 * tx + AHALO + i] * (ps.v[i] + q.v[i]);
                st4s(psout[0] + si, pn);
            }
            if (ys_tile && gy < G.ny && in_slab(gy, G.ny, G.lo[1], G.hi[1])) {
                const long long si = slab_index(G, 1, t, gy, gx);
                const F4 ps = ld4s(psin[1] + si);
                const float b = __ldg(A.cb[1] + gy);
                F4 pn;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    pn.v[i] = b * (ps.v[i] + q.v[i]);
                st4s(psout[1] + si, pn);
            }
            if (in_slab(t, G.nz, G.lo[2], G.hi[2])) {
                const long long si = slab_index(G, 2, t, gy, gx);
                const F4 ps = ld4s(psin[2] + si);
                const float b = __ldg(A.cb[2] + t);
                F4 pn;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    pn.v[i] = b * (ps.v[i] + q.v[i]);
                st4s(psout[2] + si, pn);
            }
            const F4 s = ld4s(A.s_tape + o);
            F4 gk = ld4s(A.gradK + o);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (i < nv)
                    gk.v[i] += -A.dt_over_vs * s.v[i] * apo.v[i];
            st4s(A.gradK + o, gk);
        }
        __syncthreads();
        if (tid == 0 && it + ANS < niter) {
            fence_proxy_async_smem();
            issue(it + ANS);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
            hq[j] = hq[j + 1];
    }
}

__global__ void __launch_bounds__(NTHREADS, 2)
    adj_tiled_b_kernel(const __grid_constant__ CUtensorMap mVX, const __grid_constant__ CUtensorMap mVY,
                       const __grid_constant__ CUtensorMap mVZq, const AdjTiledArgs A)
{
    using L = AdjSmemB;
    extern __shared__ __align__(1024) float sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L::END);
    const Geom &G = A.g;
    const int tid = threadIdx.x, tx = tid % (TX / 4), ty = tid / (TX / 4);
    const int tile = blockIdx.x;
    const int x0 = (tile % A.tiles_x) * TX, y0 = (tile / A.tiles_x) * TY;
    const int z0 = blockIdx.y * A.zchunk, z1 = min(G.nz, z0 + A.zchunk);
    const int shot = blockIdx.z;
    const int gx = x0 + 4 * tx, gy = y0 + ty;
    const bool row_ok = gy < G.ny && gx < G.nxp;
    const int niter = z1 - z0 + 8;
    const float w[4] = {A.c[0], A.c[1], A.c[2], A.c[3]};
    const float ndtr = -A.dtr;
    const long long fo = (long long)shot * G.vol;
    const int nv = G.nx - gx;
    const float *psin[3];
    float *psout[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        psin[d] = A.apsiv_in[d] + (long long)shot * G.slab[d];
        psout[d] = A.apsiv_out[d] + (long long)shot * G.slab[d];
    }
    const bool xs_tile = G.w[0] > 0 && (x0 - AHALO < G.lo[0] || x0 + TX + AHALO > G.nx - G.hi[0]);
    const bool ys_tile = G.w[1] > 0 && (y0 - AHALO < G.lo[1] || y0 + TY + AHALO > G.ny - G.hi[1]);
    float *cx = sm + L::CX;
    load_cx(cx, A, x0);

    if (tid == 0) {
        prefetch_tmap(&mVX);
        prefetch_tmap(&mVY);
        prefetch_tmap(&mVZq);
        for (int s = 0; s < ANS; ++s)
            mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int it) {
        const int t = z0 - 8 + it;
        float *S = sm + (it % ANS) * L::STAGE;
        uint64_t *b = &bar[it % ANS];
        const bool q_on = t + 4 >= 0 && t + 4 < G.nz, main_on = t >= z0;
        uint32_t bytes = (q_on ? TY * TX * 4u : 0u) + (main_on ? (TY * AW + AHT * TX) * 4u : 0u);
        mbar_arrive_expect_tx(b, bytes);
        if (q_on)
            tma_load_4d(S + L::VZQ, &mVZq, b, x0, y0, t + 4, shot);
        if (main_on) {
            tma_load_4d(S + L::VX, &mVX, b, x0 - AHALO, y0, t, shot);
            tma_load_4d(S + L::VY, &mVY, b, x0, y0 - AHALO, t, shot);
        }
    };
    if (tid == 0)
        for (int i = 0; i < ANS && i < niter; ++i)
            issue(i);

    F4 gq[9];   // lam_g_z(t - 4 + j)
#pragma unroll
    for (int j = 0; j < 9; ++j)
        gq[j] = f4z();

    for (int it = 0; it < niter; ++it) {
        const int t = z0 - 8 + it;
        const float *S = sm + (it % ANS) * L::STAGE;
        const bool ok = mbar_wait_bounded(&bar[it % ANS], (it / ANS) & 1, WAIT_LIMIT);

        F4 gn = f4z();
        const int zq = t + 4;
        if (ok && zq >= 0 && zq < G.nz) {
            const F4 v = ld4s(S + L::VZQ + ty * TX + 4 * tx);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                gn.v[i] = ndtr * v.v[i];
            if (row_ok && in_slab(zq, G.nz, G.lo[2], G.hi[2])) {
                const long long si = slab_index(G, 2, zq, gy, gx);
                const F4 ps = ld4s(psin[2] + si);
                const float b = __ldg(A.cb[2] + zq);
                if (zq >= z0 && zq < z1) {   // own node: update the memory variable once
                    F4 pn;
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        pn.v[i] = b * (ps.v[i] + gn.v[i]);
                    st4s(psout[2] + si, pn);
                }
                gn = corr_uniform(gn, ps, __ldg(A.ca[2] + zq), __ldg(A.ck[2] + zq));
            }
        }
        gq[8] = gn;

        const bool active = t >= z0;
        if (ok && active) {
            float *GX = sm + L::GX, *GY = sm + L::GY;
            for (int v = tid; v < TY * AW / 4; v += NTHREADS) {
                const int r = v / (AW / 4), c = 4 * (v % (AW / 4));
                F4 g = ld4s(S + L::VX + r * AW + c);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    g.v[i] *= ndtr;
                if (xs_tile)
                    corr_x(g, G, psin[0], cx, c, t, y0 + r, x0 - AHALO + c);
                st4s(GX + r * AW + c, g);
            }
            for (int v = tid; v < AHT * TX / 4; v += NTHREADS) {
                const int r = v / (TX / 4), c = 4 * (v % (TX / 4));
                F4 g = ld4s(S + L::VY + r * TX + c);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    g.v[i] *= ndtr;
                const int y = y0 - AHALO + r;
                if (ys_tile && y >= 0 && y < G.ny && x0 + c < G.nxp && in_slab(y, G.ny, G.lo[1], G.hi[1]))
                    g = corr_uniform(g, ld4s(psin[1] + slab_index(G, 1, t, y, x0 + c)), __ldg(A.ca[1] + y),
                                     __ldg(A.ck[1] + y));
                st4s(GY + r * TX + c, g);
            }
        }
        if (__syncthreads_or(ok ? 0 : 1)) {
            if (tid == 0) {
                atomicOr(A.err, ERR_TIMEOUT);
                for (int j = it; j < niter && j < it + ANS; ++j)
                    mbar_wait_bounded(&bar[j % ANS], (j / ANS) & 1, WAIT_LIMIT_DRAIN);
            }
            return;
        }
        if (active && row_ok) {
            const long long o = fo + (long long)t * G.plane + (long long)gy * G.nxp + gx;
            const F4 d1 = drow(sm + L::GX + ty * AW, 4 * tx + AHALO, w);
            const F4 d2 = dcol(sm + L::GY, TX, ty + AHALO, 4 * tx, w);
            const F4 d3 = dq(gq, w);
            F4 p = ld4s(A.ap + o);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (i < nv)
                    p.v[i] -= d1.v[i] + d2.v[i] + d3.v[i];
            st4s(A.ap + o, p);
            // own memory variables of x and y: psi <- b (psi + r)
            if (xs_tile && gy < G.ny && gx < G.nx && (gx < G.lo[0] || gx + 3 >= G.nx - G.hi[0])) {
                const long long si = slab_index(G, 0, t, gy, gx);
                const F4 ps = ld4s(psin[0] + si), v = ld4s(S + L::VX + ty * AW + 4 * tx + AHALO);
                F4 pn;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    pn.v[i] = cx[4 * tx + AHALO + i] * (ps.v[i] + ndtr * v.v[i]);
                st4s(psout[0] + si, pn);
            }
            if (ys_tile && gy < G.ny && in_slab(gy, G.ny, G.lo[1], G.hi[1])) {
                const long long si = slab_index(G, 1, t, gy, gx);
                const F4 ps = ld4s(psin[1] + si), v = ld4s(S + L::VY + (ty + AHALO) * TX + 4 * tx);
                const float b = __ldg(A.cb[1] + gy);
                F4 pn;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    pn.v[i] = b * (ps.v[i] + ndtr * v.v[i]);
                st4s(psout[1] + si, pn);
            }
        }
        __syncthreads();
        if (tid == 0 && it + ANS < niter) {
            fence_proxy_async_smem();
            issue(it + ANS);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
            gq[j] = gq[j + 1];
    }
}

// One adjoint step on the current adjoint state with the tiled kernels
// (flips the memory-variable ping-pong).
cudaError_t adjoint_step_tiled(fdtd_ctx *c, const float *s_tape)
{
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(adj_tiled_a_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             AdjSmemA::BYTES);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(adj_tiled_b_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, AdjSmemB::BYTES);
        if (e != cudaSuccess)
            return e;
        attr_done = true;
    }
    AdjTiledArgs a;
    a.g = c->g;
    a.tiles_x = c->tiles_x;
    a.zchunk = c->zchunk;
    a.kdt = c->kdt;
    a.ap = c->ap;
    const int nmax = max(c->g.nx, max(c->g.ny, c->g.nz));
    for (int d = 0; d < 3; ++d) {
        a.av[d] = c->av[d];
        a.apsiv_in[d] = c->apsiv[d][c->acur];
        a.apsiv_out[d] = c->apsiv[d][c->acur ^ 1];
        a.apsip_in[d] = c->apsip[d][c->acur];
        a.apsip_out[d] = c->apsip[d][c->acur ^ 1];
        a.cb[d] = c->coef + (d * 3 + 0) * nmax;
        a.ca[d] = c->coef + (d * 3 + 1) * nmax;
        a.ck[d] = c->coef + (d * 3 + 2) * nmax;
    }
    for (int l = 0; l < 4; ++l)
        a.c[l] = (float)(kWeights[l] / c->d.h);
    a.dtr = (float)(c->d.dt * c->vscale);
    a.dt_over_vs = (float)(c->d.dt / c->vscale);
    a.s_tape = s_tape;
    a.gradK = c->gradK;
    a.err = c->err;
    dim3 grid(c->tiles_x * c->tiles_y, c->nzchunks, c->d.nshots);
    adj_tiled_a_kernel<<<grid, NTHREADS, AdjSmemA::BYTES, c->stream>>>(c->amaps[0], c->amaps[1], c->amaps[2],
                                                                        c->mapK, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    adj_tiled_b_kernel<<<grid, NTHREADS, AdjSmemB::BYTES, c->stream>>>(c->amaps[3], c->amaps[4], c->amaps[5], a);
    e = cudaGetLastError();
    c->acur ^= 1;
    return e;
}

}  // namespace fdtd

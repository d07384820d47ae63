// Discrete adjoint of one time step as one fused z-march kernel, the mirror
// image of the forward step kernel (paper Sec. 3.1-3.2 transposed; the
// assignment-by-assignment transpose is spelled out in fdtd_adjoint.cu):
//
//   stage A (transpose of the pressure update), per node:
//     q = kr_d kdt lam_p                         (kdt = -dt K / vscale; kr_d the
//                                                 anisotropy factor of axis d, 1 if none)
//     lam_h_d = q + [d-slab] ((kinv_d - 1) q + a_d (lam_psip_d + q))
//     lam_v'_d = lam_v_d - D_d lam_h_d ;  lam_psip_d <- b_d (lam_psip_d + q)
//     dJ/dK += -(dt / vscale) S lam_p            (S: the taped bracket)
//   stage B (transpose of the velocity update), per node:
//     r_d = -dtr lam_v'_d                        (-dtr / rho with a density)
//     lam_g_d = r_d + [d-slab] ((kinv_d - 1) r_d + a_d (lam_psiv_d + r_d))
//     lam_p' = lam_p - sum_d D_d lam_g_d ;  lam_psiv_d <- b_d (lam_psiv_d + r_d)
//
// Per CTA: a 32 x 32 tile in (x, y), a z range marched plane by plane.  At
// plane t the CTA forms lam_h_x / lam_h_y over the tile with an 8-node halo
// (from lam_p and kdt staged by TMA with that halo) in shared memory, then
// lam_v' on the tile and its 4-node halo (the halo recomputed, not stored),
// and from it lam_g in shared memory, then lam_p' on the tile.  Along z,
// lam_h_z runs 8 planes ahead and lam_g_z 4 planes ahead in 9-plane register
// queues.  The adjoint pressure is kept as mu = kdt lam_p, the quantity
// stage A differentiates (lam_h = mu outside the slabs), so the CTAs away
// from the slabs differentiate the staged mu plane directly.  mu and lam_v
// are read from one set and written to the other; so are the memory
// variables.  One pass reads mu, lam_v, kdt, the tape and dJ/dK and writes
// mu, lam_v and dJ/dK (48 B per node and shot, FP32: 7 words read, 5 written),
// plus the slab memory variables (16 B per slab node and axis).
#include "fdtd_internal.cuh"

namespace fdtd {

namespace {

constexpr int AH = 8;                 // lam_h halo
constexpr int AW = TX + 2 * AH;       // 48
constexpr int ANS = 3;                // TMA stages
constexpr int GW = TX + 8;            // lam_g rows: x0 - 4 .. x0 + TX + 4

struct FusedLayout {
    // one stage (floats)
    static constexpr int P = 0;                    // mu      [48][48] at (x0-8, y0-8, t)
    static constexpr int PQ = P + AW * AW;         // mu      [32][32] at t+8
    static constexpr int VX = PQ + TY * TX;        // lam_v_x [32][40] at (x0-4, y0, t)
    static constexpr int VY = VX + TY * GW;        // lam_v_y [40][32] at (x0, y0-4, t)
    static constexpr int VZ = VY + GW * TX;        // lam_v_z [32][32] at t+4
    static constexpr int KT = VZ + TY * TX;        // kdt     [32][32] at t
    static constexpr int STAGE = KT + TY * TX;
    // work region after the stages: lam_h_x [32][48] and lam_h_y [48][32]
    // (CTAs that meet a slab), then lam_g_x [32][40] and lam_g_y [40][32]
    static constexpr int W = ANS * STAGE;
    static constexpr int HX = W, HY = W + TY * AW;
    static constexpr int GX = W, GY = W + TY * GW;
    static constexpr int CX = W + 2 * TY * AW;     // b, a, 1/kappa over x0-8 .. x0+40
    static constexpr int CY = CX + 3 * AW;         // same over y
    static constexpr int CXV = CY + 3 * AW;        // the velocity profiles (half nodes when staggered)
    static constexpr int CYV = CXV + 3 * AW;
    static constexpr int END = CYV + 3 * AW;
    static constexpr int BYTES = END * 4 + 8 * ANS;
    static_assert((PQ * 4) % 128 == 0 && (VX * 4) % 128 == 0 && (VY * 4) % 128 == 0 && (VZ * 4) % 128 == 0 &&
                      (KT * 4) % 128 == 0 && (STAGE * 4) % 128 == 0,
                  "TMA destinations must stay 128-byte aligned");
    static_assert(2 * TY * GW <= 2 * TY * AW, "lam_g fits in the lam_h region");
};

struct FusedArgs {
    Geom g;
    int tiles_x;
    int zmid0, zmid1, zchunk;          // chunks: [0, zmid0), zchunk planes over [zmid0, zmid1), [zmid1, nz)
    const float *kdt;                  // [vol]
    const float *ap_in;                // mu = kdt lam_p, [nshots][vol]
    float *ap_out;
    const float *av_in[3];
    float *av_out[3];
    const float *apsiv_in[3];
    float *apsiv_out[3];
    const float *apsip_in[3];
    float *apsip_out[3];
    const float *cb[3], *ca[3], *ck[3];
    const float *cbv[3], *cav[3], *ckv[3];   // velocity profiles (half nodes when staggered, else cb..)
    float c[4];
    float dtr;
    float dt_over_vs;
    float kr[3];                       // anisotropy factors of the pressure bracket (x, y, z)
    const float *nbr;                  // density: -dtr / rho per node [vol] (the forward's table)
    const float *lb[3], *la[3];        // local grading: b, a per slab node (slab layout), or null
    const float *s_tape;               // [nshots][vol]
    float *gradK;                      // [nshots][vol]
    unsigned *err;
};

__host__ __device__ __forceinline__ int adj_chunks(const FusedArgs &A)
{
    return (A.zmid0 > 0 ? 1 : 0) + (A.zmid1 - A.zmid0 + A.zchunk - 1) / A.zchunk + (A.g.nz > A.zmid1 ? 1 : 0);
}

// long middle chunks first, the end chunks last
__device__ __forceinline__ void adj_chunk_range(const FusedArgs &A, int y, int *z0, int *z1)
{
    const int nmid = (A.zmid1 - A.zmid0 + A.zchunk - 1) / A.zchunk;
    if (y < nmid) {
        *z0 = A.zmid0 + y * A.zchunk;
        *z1 = min(A.zmid1, *z0 + A.zchunk);
    } else if (y == nmid && A.zmid0 > 0) {
        *z0 = 0;
        *z1 = A.zmid0;
    } else {
        *z0 = A.zmid1;
        *z1 = A.g.nz;
    }
}

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
__device__ __forceinline__ float2 ld2s(const float *p) { return *reinterpret_cast<const float2 *>(p); }

// D along a row: outputs at columns c0 .. c0+3 of `row` (c0 - 4 >= 0, c0 % 4 == 0)
// Stencil modes: 0 centred (offsets +l, -l); 1 staggered forward, node ->
// half node (+l, 1-l); 2 staggered backward, half node -> node (l-1, -l).
template <int M>
__host__ __device__ constexpr int offp(int l) { return M == 2 ? l - 1 : l; }
template <int M>
__host__ __device__ constexpr int offm(int l) { return M == 1 ? 1 - l : -l; }

template <int M>
__device__ __forceinline__ F4 drow(const float *row, int c0, const float *w)
{
    const F4 a = ld4s(row + c0 - 4), b = ld4s(row + c0), c = ld4s(row + c0 + 4);
    const float f[12] = {a.v[0], a.v[1], a.v[2], a.v[3], b.v[0], b.v[1], b.v[2], b.v[3], c.v[0], c.v[1], c.v[2], c.v[3]};
    F4 r;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        r.v[i] = w[0] * (f[i + 4 + offp<M>(1)] - f[i + 4 + offm<M>(1)]) +
                 w[1] * (f[i + 4 + offp<M>(2)] - f[i + 4 + offm<M>(2)]) +
                 w[2] * (f[i + 4 + offp<M>(3)] - f[i + 4 + offm<M>(3)]) +
                 w[3] * (f[i + 4 + offp<M>(4)] - f[i + 4 + offm<M>(4)]);
    return r;
}

// the same for one pair of outputs at columns c0, c0+1 (c0 even, c0 - 4 >= 0)
template <int M>
__device__ __forceinline__ float2 drow2(const float *row, int c0, const float *w)
{
    float f[10];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float2 v = ld2s(row + c0 - 4 + 2 * k);
        f[2 * k] = v.x;
        f[2 * k + 1] = v.y;
    }
    float o[2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
        o[i] = w[0] * (f[i + 4 + offp<M>(1)] - f[i + 4 + offm<M>(1)]) +
               w[1] * (f[i + 4 + offp<M>(2)] - f[i + 4 + offm<M>(2)]) +
               w[2] * (f[i + 4 + offp<M>(3)] - f[i + 4 + offm<M>(3)]) +
               w[3] * (f[i + 4 + offp<M>(4)] - f[i + 4 + offm<M>(4)]);
    return make_float2(o[0], o[1]);
}

// D along a column of a plane with `stride`: rows r0 + offp, r0 + offm, 4 columns at c
template <int M>
__device__ __forceinline__ F4 dcol(const float *plane, int stride, int r0, int c, const float *w)
{
    F4 r = f4z();
#pragma unroll
    for (int l = 1; l <= 4; ++l) {
        const F4 p = ld4s(plane + (r0 + offp<M>(l)) * stride + c), m = ld4s(plane + (r0 + offm<M>(l)) * stride + c);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            r.v[i] += w[l - 1] * (p.v[i] - m.v[i]);
    }
    return r;
}

template <int M>
__device__ __forceinline__ float2 dcol2(const float *plane, int stride, int r0, int c, const float *w)
{
    float2 r = make_float2(0.f, 0.f);
#pragma unroll
    for (int l = 1; l <= 4; ++l) {
        const float2 p = ld2s(plane + (r0 + offp<M>(l)) * stride + c), m = ld2s(plane + (r0 + offm<M>(l)) * stride + c);
        r.x += w[l - 1] * (p.x - m.x);
        r.y += w[l - 1] * (p.y - m.y);
    }
    return r;
}

// D_z at the centre of a 9-plane queue
template <int M>
__device__ __forceinline__ F4 dq(const F4 *q, const float *w)
{
    F4 r;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        r.v[i] = w[0] * (q[4 + offp<M>(1)].v[i] - q[4 + offm<M>(1)].v[i]) +
                 w[1] * (q[4 + offp<M>(2)].v[i] - q[4 + offm<M>(2)].v[i]) +
                 w[2] * (q[4 + offp<M>(3)].v[i] - q[4 + offm<M>(3)].v[i]) +
                 w[3] * (q[4 + offp<M>(4)].v[i] - q[4 + offm<M>(4)].v[i]);
    return r;
}

__device__ __forceinline__ F4 f4s(float a) { return F4{{a, a, a, a}}; }
// per-node coefficients of 4 nodes (local grading tables, read-only)
__device__ __forceinline__ F4 ldc4(const float *p) { return Io<float>::ldg4(p); }
__device__ __forceinline__ float2 ldc2(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }

// lam + ((kinv - 1) lam + a (psi + lam)): the CPML bracket's transpose
__device__ __forceinline__ float corr1(float lam, float psi, float a, float k)
{
    return lam + (k - 1.f) * lam + a * (psi + lam);
}

// Own-node store of a full field; lanes beyond nx keep their value.
__device__ __forceinline__ void st_own(float *p, const F4 &v, int nv)
{
    if (nv >= 4) {
        st4s(p, v);
        return;
    }
    F4 o = ld4s(p);
#pragma unroll
    for (int i = 0; i < 4; ++i)
        o.v[i] = i < nv ? v.v[i] : o.v[i];
    st4s(p, o);
}

// The body of one CTA.  kEdge = false: the tile with its 8-node x / y halo
// and the z range with 8 planes either side lie inside the grid and outside
// every CPML slab; then lam_h = mu, and the derivatives of stage A read the
// staged mu plane directly.  kEdge = true forms lam_h in shared memory first.
// kRho: the velocity transpose takes -dtr / rho per node from A.nbr.
// kLocal: b and a of every slab node come from A.lb, A.la (local grading).
// kStag: the staggered form's transpose: stage A applies D+ to lam_h, stage B
// D- to lam_g, and the velocity transpose takes the half-node profiles.
template <bool kEdge, bool kRho, bool kLocal, bool kStag>
__device__ __forceinline__ void adj_body(const CUtensorMap &mP, const CUtensorMap &mPq, const CUtensorMap &mVX,
                                         const CUtensorMap &mVY, const CUtensorMap &mVZ, const CUtensorMap &mK,
                                         const FusedArgs &A, int z0, int z1, float *sm)
{
    using L = FusedLayout;
    constexpr int kSA = kStag ? 1 : 0, kSB = kStag ? 2 : 0;   // stencil modes of stages A and B
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L::END);
    float *HX = sm + L::HX, *HY = sm + L::HY, *GX = sm + L::GX, *GY = sm + L::GY;
    float *sCx = sm + L::CX, *sCy = sm + L::CY;   // [3][48]: b, a, 1/kappa
    float *sCxv = kStag ? sm + L::CXV : sCx, *sCyv = kStag ? sm + L::CYV : sCy;   // velocity transpose
    const Geom &G = A.g;
    const int tid = threadIdx.x, tx = tid % (TX / 4), ty = tid / (TX / 4);
    const int tile = blockIdx.x;
    const int x0 = (tile % A.tiles_x) * TX, y0 = (tile / A.tiles_x) * TY;
    const int shot = blockIdx.z;
    const int gx = x0 + 4 * tx, gy = y0 + ty;
    const bool row_ok = gy < G.ny && gx < G.nxp;
    const int nv = G.nx - gx;   // lanes of this thread inside the grid
    const int niter = z1 - z0 + 8;
    const float w[4] = {A.c[0], A.c[1], A.c[2], A.c[3]};
    const float ndtr = -A.dtr;
    const long long fo = (long long)shot * G.vol;
    const long long rowofs = (long long)gy * G.nxp + gx;
    const float *psvin[3], *pspin[3];
    float *psvout[3], *pspout[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        psvin[d] = A.apsiv_in[d] + (long long)shot * G.slab[d];
        psvout[d] = A.apsiv_out[d] + (long long)shot * G.slab[d];
        pspin[d] = A.apsip_in[d] + (long long)shot * G.slab[d];
        pspout[d] = A.apsip_out[d] + (long long)shot * G.slab[d];
    }
    const bool xs_tile = kEdge && G.w[0] > 0 && (x0 - AH < G.lo[0] || x0 + TX + AH > G.nx - G.hi[0]);
    const bool ys_tile = kEdge && G.w[1] > 0 && (y0 - AH < G.lo[1] || y0 + TY + AH > G.ny - G.hi[1]);
    const bool own_x = xs_tile && gy < G.ny && gx < G.nx && (gx < G.lo[0] || gx + 3 >= G.nx - G.hi[0]);
    const bool own_y = ys_tile && row_ok && in_slab(gy, G.ny, G.lo[1], G.hi[1]);

    for (int i = tid; kEdge && i < 3 * AW; i += NTHREADS) {
        const int c = i / AW, x = x0 - AH + i % AW, y = y0 - AH + i % AW;
        const bool inx = x >= 0 && x < G.nx && in_slab(x, G.nx, G.lo[0], G.hi[0]);
        const bool iny = y >= 0 && y < G.ny && in_slab(y, G.ny, G.lo[1], G.hi[1]);
        sCx[i] = inx ? (c == 0 ? A.cb[0][x] : (c == 1 ? A.ca[0][x] : A.ck[0][x])) : (c == 2 ? 1.f : 0.f);
        sCy[i] = iny ? (c == 0 ? A.cb[1][y] : (c == 1 ? A.ca[1][y] : A.ck[1][y])) : (c == 2 ? 1.f : 0.f);
        if (kStag) {
            sCxv[i] = inx ? (c == 0 ? A.cbv[0][x] : (c == 1 ? A.cav[0][x] : A.ckv[0][x])) : (c == 2 ? 1.f : 0.f);
            sCyv[i] = iny ? (c == 0 ? A.cbv[1][y] : (c == 1 ? A.cav[1][y] : A.ckv[1][y])) : (c == 2 ? 1.f : 0.f);
        }
    }

    // halo task: one pair of nodes.  Threads 0..127: lam_v'_y on the y halo
    // (8 rows x 16 pairs), 128..255: lam_v'_x on the x halo (32 rows x 4 pairs)
    const bool do_yhalo = tid < 128;
    const int yh_r = (tid / 16) & 7;
    const int yh_y = yh_r < 4 ? y0 - 4 + yh_r : y0 + TY + (yh_r - 4);
    const int yh_x = x0 + 2 * (tid % 16);
    const int xh_k = tid & 3;
    const int xh_x = xh_k < 2 ? x0 - 4 + 2 * xh_k : x0 + TX + 2 * (xh_k - 2);
    const int xh_y = y0 + ((tid - 128) >> 2);
    const bool yh_in = do_yhalo && yh_y >= 0 && yh_y < G.ny;
    const bool xh_in = !do_yhalo && xh_y < G.ny;

    if (tid == 0) {
        prefetch_tmap(&mP);
        prefetch_tmap(&mPq);
        prefetch_tmap(&mVX);
        prefetch_tmap(&mVY);
        prefetch_tmap(&mVZ);
        prefetch_tmap(&mK);
        for (int s = 0; s < ANS; ++s)
            mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int it) {
        const int t = z0 - 8 + it;
        float *S = sm + (it % ANS) * L::STAGE;
        uint64_t *b = &bar[it % ANS];
        const bool q_on = t + 8 >= 0 && t + 8 < G.nz;
        const bool vz_on = t + 4 >= 0 && t + 4 < G.nz;
        const bool main_on = t >= z0;
        uint32_t bytes = (q_on ? TY * TX * 4u : 0u) + (vz_on ? TY * TX * 4u : 0u) +
                         (main_on ? (AW * AW + 2u * TY * GW + TY * TX) * 4u : 0u);
        mbar_arrive_expect_tx(b, bytes);
        if (q_on)
            tma_load_4d(S + L::PQ, &mPq, b, x0, y0, t + 8, shot);
        if (vz_on)
            tma_load_4d(S + L::VZ, &mVZ, b, x0, y0, t + 4, shot);
        if (main_on) {
            tma_load_4d(S + L::P, &mP, b, x0 - AH, y0 - AH, t, shot);
            tma_load_4d(S + L::VX, &mVX, b, x0 - 4, y0, t, shot);
            tma_load_4d(S + L::VY, &mVY, b, x0, y0 - 4, t, shot);
            tma_load_3d(S + L::KT, &mK, b, x0, y0, t);
        }
    };
    if (tid == 0)
        for (int i = 0; i < ANS && i < niter; ++i)
            issue(i);

    // queues: hq[j] = lam_h_z(t + j), gq[j] = lam_g_z(t - 4 + j)
    F4 hq[9], gq[9];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int z = z0 - 8 + k;
        hq[k] = f4z();
        gq[k] = f4z();
        if (z >= 0 && row_ok) {
            hq[k] = ld4s(A.ap_in + fo + (long long)z * G.plane + rowofs);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                hq[k].v[i] *= A.kr[2];
            if (kEdge && in_slab(z, G.nz, G.lo[2], G.hi[2])) {
                const long long si = slab_index(G, 2, z, gy, gx);
                const F4 ps = ld4s(pspin[2] + si);
                const F4 a = kLocal ? ldc4(A.la[2] + si) : f4s(__ldg(A.ca[2] + z));
                const float kk = __ldg(A.ck[2] + z);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    hq[k].v[i] = corr1(hq[k].v[i], ps.v[i], a.v[i], kk);
            }
        }
    }
    hq[8] = f4z();
    gq[8] = f4z();

    for (int it = 0; it < niter; ++it) {
        const int t = z0 - 8 + it;
        const bool active = t >= z0;
        const float *S = sm + (it % ANS) * L::STAGE;
        if (active && row_ok && t + 1 < z1) {
            const long long on = fo + (long long)(t + 1) * G.plane + rowofs;
            prefetch_l2(A.s_tape + on);
            prefetch_l2(A.gradK + on);
        }
        // memory variables of the next plane into L2 (CTAs that meet a slab)
        if (kEdge && t + 1 >= z0 && t + 1 < z1) {
            const int tn = t + 1;
            if (xs_tile || ys_tile) {
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const int v = tid + j * NTHREADS;
                    if (v < TY * AW / 4) {
                        const int r = v / (AW / 4), c = 4 * (v % (AW / 4)), x = x0 - AH + c, y = y0 + r;
                        if (xs_tile && x >= 0 && x < G.nx && y < G.ny && (x < G.lo[0] || x + 3 >= G.nx - G.hi[0]))
                            prefetch_l2(pspin[0] + slab_index(G, 0, tn, y, x));
                    } else {
                        const int u = v - TY * AW / 4, r = u / (TX / 4), c = 4 * (u % (TX / 4));
                        const int y = y0 - AH + r, x = x0 + c;
                        if (ys_tile && y >= 0 && y < G.ny && x < G.nxp && in_slab(y, G.ny, G.lo[1], G.hi[1]))
                            prefetch_l2(pspin[1] + slab_index(G, 1, tn, y, x));
                    }
                }
            }
            if (own_x)
                prefetch_l2(psvin[0] + slab_index(G, 0, tn, gy, gx));
            if (own_y)
                prefetch_l2(psvin[1] + slab_index(G, 1, tn, gy, gx));
            if (do_yhalo && ys_tile && yh_in && yh_x < G.nxp && in_slab(yh_y, G.ny, G.lo[1], G.hi[1]))
                prefetch_l2(psvin[1] + slab_index(G, 1, tn, yh_y, yh_x));
            if (!do_yhalo && xs_tile && xh_in && xh_x >= 0 && xh_x < G.nx &&
                (xh_x < G.lo[0] || xh_x + 1 >= G.nx - G.hi[0]))
                prefetch_l2(psvin[0] + slab_index(G, 0, tn, xh_y, xh_x));
        }
        if (kEdge && row_ok) {
            const int zq = t + 9, zv = t + 5;
            if (zq < G.nz && in_slab(zq, G.nz, G.lo[2], G.hi[2]))
                prefetch_l2(pspin[2] + slab_index(G, 2, zq, gy, gx));
            if (zv >= 0 && zv < G.nz && in_slab(zv, G.nz, G.lo[2], G.hi[2]))
                prefetch_l2(psvin[2] + slab_index(G, 2, zv, gy, gx));
        }
        const bool ok = mbar_wait_bounded(&bar[it % ANS], (it / ANS) & 1, WAIT_LIMIT);

        // ---- z block: lam_h_z at t + 8, lam_v'_z and lam_g_z at t + 4, D_z lam_g_z at t
        {
            const int zq = t + 8;
            F4 hn = f4z();
            if (ok && zq >= 0 && zq < G.nz) {
                hn = ld4s(S + L::PQ + ty * TX + 4 * tx);   // TMA fills zeros beyond the grid
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    hn.v[i] *= A.kr[2];
                if (kEdge && row_ok && in_slab(zq, G.nz, G.lo[2], G.hi[2])) {
                    const long long si = slab_index(G, 2, zq, gy, gx);
                    const F4 ps = ld4s(pspin[2] + si);
                    const F4 a = kLocal ? ldc4(A.la[2] + si) : f4s(__ldg(A.ca[2] + zq));
                    const float kk = __ldg(A.ck[2] + zq);
                    if (zq >= z0 && zq < z1) {
                        const F4 b = kLocal ? ldc4(A.lb[2] + si) : f4s(__ldg(A.cb[2] + zq));
                        F4 pn;
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            pn.v[i] = b.v[i] * (ps.v[i] + hn.v[i]);
                        st4s(pspout[2] + si, pn);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        hn.v[i] = corr1(hn.v[i], ps.v[i], a.v[i], kk);
                }
            }
            hq[8] = hn;
            const int zv = t + 4;
            F4 gn = f4z();
            if (ok && zv >= 0 && zv < G.nz) {
                const F4 dh = dq<kSA>(hq, w);
                F4 vz = ld4s(S + L::VZ + ty * TX + 4 * tx);
                F4 fz = F4{{ndtr, ndtr, ndtr, ndtr}};
                if (kRho)
                    fz = row_ok ? Io<float>::ldg4(A.nbr + (long long)zv * G.plane + rowofs) : f4z();
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    vz.v[i] -= dh.v[i];
                    gn.v[i] = fz.v[i] * vz.v[i];
                }
                const bool owned = zv >= z0 && zv < z1;
                if (owned && row_ok)
                    st_own(A.av_out[2] + fo + (long long)zv * G.plane + rowofs, vz, nv);
                if (kEdge && row_ok && in_slab(zv, G.nz, G.lo[2], G.hi[2])) {
                    const long long si = slab_index(G, 2, zv, gy, gx);
                    const F4 ps = ld4s(psvin[2] + si);
                    if (owned) {
                        const F4 b = kLocal ? ldc4(A.lb[2] + si) : f4s(__ldg(A.cbv[2] + zv));
                        F4 pn;
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            pn.v[i] = b.v[i] * (ps.v[i] + gn.v[i]);
                        st4s(psvout[2] + si, pn);
                    }
                    const F4 a = kLocal ? ldc4(A.la[2] + si) : f4s(__ldg(A.cav[2] + zv));
                    const float kk = __ldg(A.ckv[2] + zv);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        gn.v[i] = corr1(gn.v[i], ps.v[i], a.v[i], kk);
                }
            }
            gq[8] = gn;
        }
        const F4 hz = dq<kSB>(gq, w);

        // sources of D_x lam_h_x (row r <-> y0 + r, column c <-> x0 - 8 + c)
        // and D_y lam_h_y (row r <-> y0 - 8 + r, column c <-> x0 + c): shared
        // memory where the tile meets an x (y) slab, else the staged mu plane
        const float *hxs = xs_tile ? HX : S + L::P + AH * AW;
        const float *hys = ys_tile ? HY : S + L::P + AH;
        constexpr int hxw = AW;
        const int hyw = ys_tile ? TX : AW;
        const bool build_h = xs_tile || ys_tile;   // CTA-uniform
        // lam_h in shared memory carries kr_d already; the staged mu plane
        // does not, so derivatives read from it are scaled by kr_d
        const float kxs = xs_tile ? 1.f : A.kr[0], kys = ys_tile ? 1.f : A.kr[1];

        if (kEdge) {
            // ---- lam_h_x (own rows, x halo 8), lam_h_y (own columns, y halo 8)
            if (ok && active && build_h) {
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const int v = tid + j * NTHREADS;   // 0 .. 767
                    if (v < TY * AW / 4) {
                        if (!xs_tile)
                            continue;
                        const int r = v / (AW / 4), c = 4 * (v % (AW / 4));
                        F4 h = ld4s(S + L::P + (r + AH) * AW + c);
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            h.v[i] *= A.kr[0];
                        const int x = x0 - AH + c, y = y0 + r;
                        if (xs_tile && x >= 0 && x < G.nx && y < G.ny && (x < G.lo[0] || x + 3 >= G.nx - G.hi[0])) {
                            const long long si = slab_index(G, 0, t, y, x);
                            const F4 ps = ld4s(pspin[0] + si);
                            const F4 a = kLocal ? ldc4(A.la[0] + si)
                                                : F4{{sCx[AW + c], sCx[AW + c + 1], sCx[AW + c + 2], sCx[AW + c + 3]}};
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                h.v[i] = corr1(h.v[i], ps.v[i], a.v[i], sCx[2 * AW + c + i]);
                        }
                        st4s(HX + r * AW + c, h);
                    } else {
                        if (!ys_tile)
                            continue;
                        const int u = v - TY * AW / 4;  // 0 .. 383
                        const int r = u / (TX / 4), c = 4 * (u % (TX / 4));
                        F4 h = ld4s(S + L::P + r * AW + c + AH);
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            h.v[i] *= A.kr[1];
                        const int y = y0 - AH + r, x = x0 + c;
                        if (ys_tile && y >= 0 && y < G.ny && x < G.nxp && in_slab(y, G.ny, G.lo[1], G.hi[1])) {
                            const long long si = slab_index(G, 1, t, y, x);
                            const F4 ps = ld4s(pspin[1] + si);
                            const F4 a = kLocal ? ldc4(A.la[1] + si) : f4s(sCy[AW + r]);
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                h.v[i] = corr1(h.v[i], ps.v[i], a.v[i], sCy[2 * AW + r]);
                        }
                        st4s(HY + r * TX + c, h);
                    }
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
        }

        // ---- lam_v' on own nodes and the halo pair; lam_g kept in registers
        F4 gxo = f4z(), gyo = f4z();
        float2 gh = make_float2(0.f, 0.f);
        if (ok && active) {
            const long long o = fo + (long long)t * G.plane + rowofs;
            F4 fo4 = F4{{ndtr, ndtr, ndtr, ndtr}};
            if (kRho)
                fo4 = row_ok ? Io<float>::ldg4(A.nbr + (long long)t * G.plane + rowofs) : f4z();
            {
                F4 vx = ld4s(S + L::VX + ty * GW + 4 * tx + 4);
                const F4 dh = drow<kSA>(hxs + ty * hxw, 4 * tx + AH, w);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    vx.v[i] -= kxs * dh.v[i];
                    gxo.v[i] = fo4.v[i] * vx.v[i];
                }
                if (own_x) {
                    const long long si = slab_index(G, 0, t, gy, gx);
                    const F4 ps = ld4s(psvin[0] + si);
                    const int c0 = 4 * tx + AH;
                    const F4 b = kLocal ? ldc4(A.lb[0] + si) : F4{{sCxv[c0], sCxv[c0 + 1], sCxv[c0 + 2], sCxv[c0 + 3]}};
                    const F4 a = kLocal ? ldc4(A.la[0] + si)
                                        : F4{{sCxv[AW + c0], sCxv[AW + c0 + 1], sCxv[AW + c0 + 2], sCxv[AW + c0 + 3]}};
                    F4 pn;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int cc = c0 + i;
                        pn.v[i] = b.v[i] * (ps.v[i] + gxo.v[i]);
                        gxo.v[i] = corr1(gxo.v[i], ps.v[i], a.v[i], sCxv[2 * AW + cc]);
                    }
                    st4s(psvout[0] + si, pn);
                }
                if (row_ok)
                    st_own(A.av_out[0] + o, vx, nv);
            }
            {
                F4 vy = ld4s(S + L::VY + (ty + 4) * TX + 4 * tx);
                const F4 dh = dcol<kSA>(hys, hyw, ty + AH, 4 * tx, w);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    vy.v[i] -= kys * dh.v[i];
                    gyo.v[i] = fo4.v[i] * vy.v[i];
                }
                if (own_y) {
                    const long long si = slab_index(G, 1, t, gy, gx);
                    const F4 ps = ld4s(psvin[1] + si);
                    const F4 b = kLocal ? ldc4(A.lb[1] + si) : f4s(sCyv[ty + AH]);
                    const F4 a = kLocal ? ldc4(A.la[1] + si) : f4s(sCyv[AW + ty + AH]);
                    const float kk = sCyv[2 * AW + ty + AH];
                    F4 pn;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        pn.v[i] = b.v[i] * (ps.v[i] + gyo.v[i]);
                        gyo.v[i] = corr1(gyo.v[i], ps.v[i], a.v[i], kk);
                    }
                    st4s(psvout[1] + si, pn);
                }
                if (row_ok)
                    st_own(A.av_out[1] + o, vy, nv);
            }
            if (kEdge) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    gxo.v[i] = (gy < G.ny && i < nv) ? gxo.v[i] : 0.f;
                    gyo.v[i] = (gy < G.ny && i < nv) ? gyo.v[i] : 0.f;
                }
            }
            // halo pair of lam_v' (recomputed, not stored), then lam_g
            if (do_yhalo) {
                const int r = yh_y - y0 + 4, c = yh_x - x0;
                float2 vy = ld2s(S + L::VY + r * TX + c);
                const float2 dh = dcol2<kSA>(hys, hyw, yh_y - y0 + AH, c, w);
                float2 fh = make_float2(ndtr, ndtr);
                if (kRho)
                    fh = (yh_in && yh_x < G.nxp)
                             ? __ldg(reinterpret_cast<const float2 *>(A.nbr + (long long)t * G.plane +
                                                                       (long long)yh_y * G.nxp + yh_x))
                             : make_float2(0.f, 0.f);
                gh = make_float2(fh.x * (vy.x - kys * dh.x), fh.y * (vy.y - kys * dh.y));
                if (kEdge) {
                    if (ys_tile && yh_in && yh_x < G.nxp && in_slab(yh_y, G.ny, G.lo[1], G.hi[1])) {
                        const long long ih = slab_index(G, 1, t, yh_y, yh_x);
                        const float2 ps = ld2s(psvin[1] + ih);
                        const float2 a = kLocal ? ldc2(A.la[1] + ih) : make_float2(sCyv[AW + r + 4], sCyv[AW + r + 4]);
                        const float kk = sCyv[2 * AW + r + 4];
                        gh.x = corr1(gh.x, ps.x, a.x, kk);
                        gh.y = corr1(gh.y, ps.y, a.y, kk);
                    }
                    gh.x = (yh_in && yh_x < G.nx) ? gh.x : 0.f;
                    gh.y = (yh_in && yh_x + 1 < G.nx) ? gh.y : 0.f;
                }
            } else {
                const int r = xh_y - y0, c = xh_x - x0 + 4;
                float2 vx = ld2s(S + L::VX + r * GW + c);
                const float2 dh = drow2<kSA>(hxs + r * hxw, xh_x - x0 + AH, w);
                float2 fh = make_float2(ndtr, ndtr);
                if (kRho)
                    fh = (xh_in && xh_x >= 0 && xh_x < G.nxp)
                             ? __ldg(reinterpret_cast<const float2 *>(A.nbr + (long long)t * G.plane +
                                                                       (long long)xh_y * G.nxp + xh_x))
                             : make_float2(0.f, 0.f);
                gh = make_float2(fh.x * (vx.x - kxs * dh.x), fh.y * (vx.y - kxs * dh.y));
                if (kEdge) {
                    if (xs_tile && xh_in && xh_x >= 0 && xh_x < G.nx &&
                        (xh_x < G.lo[0] || xh_x + 1 >= G.nx - G.hi[0])) {
                        const long long ih = slab_index(G, 0, t, xh_y, xh_x);
                        const float2 ps = ld2s(psvin[0] + ih);
                        const int cc = xh_x - x0 + AH;
                        const float2 a = kLocal ? ldc2(A.la[0] + ih) : make_float2(sCxv[AW + cc], sCxv[AW + cc + 1]);
                        gh.x = corr1(gh.x, ps.x, a.x, sCxv[2 * AW + cc]);
                        gh.y = corr1(gh.y, ps.y, a.y, sCxv[2 * AW + cc + 1]);
                    }
                    gh.x = (xh_in && xh_x >= 0 && xh_x < G.nx) ? gh.x : 0.f;
                    gh.y = (xh_in && xh_x + 1 >= 0 && xh_x + 1 < G.nx) ? gh.y : 0.f;
                }
            }
            // own memory variables of lam_p (x, y slabs) and dJ/dK
            if (row_ok) {
                const F4 q = ld4s(S + L::P + (ty + AH) * AW + 4 * tx + AH);   // mu = kdt lam_p
                if (own_x) {
                    const long long si = slab_index(G, 0, t, gy, gx);
                    const F4 ps = ld4s(pspin[0] + si);
                    const int c0 = 4 * tx + AH;
                    const F4 b = kLocal ? ldc4(A.lb[0] + si) : F4{{sCx[c0], sCx[c0 + 1], sCx[c0 + 2], sCx[c0 + 3]}};
                    F4 pn;
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        pn.v[i] = b.v[i] * (ps.v[i] + A.kr[0] * q.v[i]);
                    st4s(pspout[0] + si, pn);
                }
                if (own_y) {
                    const long long si = slab_index(G, 1, t, gy, gx);
                    const F4 ps = ld4s(pspin[1] + si);
                    const F4 b = kLocal ? ldc4(A.lb[1] + si) : f4s(sCy[ty + AH]);
                    F4 pn;
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        pn.v[i] = b.v[i] * (ps.v[i] + A.kr[1] * q.v[i]);
                    st4s(pspout[1] + si, pn);
                }
                const F4 kd = ld4s(S + L::KT + ty * TX + 4 * tx);
                const F4 sv = ld4s(A.s_tape + o);
                F4 gk = ld4s(A.gradK + o);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (i < nv)
                        gk.v[i] += -A.dt_over_vs * sv.v[i] * (q.v[i] / kd.v[i]);
                st4s(A.gradK + o, gk);
            }
        }
        if (kEdge && build_h)
            __syncthreads();   // the lam_h region becomes the lam_g region
        if (ok && active) {
            st4s(GX + ty * GW + 4 * tx + 4, gxo);
            st4s(GY + (ty + 4) * TX + 4 * tx, gyo);
            if (do_yhalo)
                *reinterpret_cast<float2 *>(GY + (yh_y - y0 + 4) * TX + (yh_x - x0)) = gh;
            else
                *reinterpret_cast<float2 *>(GX + (xh_y - y0) * GW + (xh_x - x0 + 4)) = gh;
        }
        if (kEdge) {
            __syncthreads();
        } else if (__syncthreads_or(ok ? 0 : 1)) {
            if (tid == 0) {
                atomicOr(A.err, ERR_TIMEOUT);
                for (int j = it; j < niter && j < it + ANS; ++j)
                    mbar_wait_bounded(&bar[j % ANS], (j / ANS) & 1, WAIT_LIMIT_DRAIN);
            }
            return;
        }

        if (active && row_ok) {
            // ---- stage B: mu' = mu - kdt (D_x lam_g_x + D_y lam_g_y + D_z lam_g_z)
            const long long o = fo + (long long)t * G.plane + rowofs;
            const F4 d1 = drow<kSB>(GX + ty * GW, 4 * tx + 4, w);
            const F4 d2 = dcol<kSB>(GY, TX, ty + 4, 4 * tx, w);
            const F4 kd = ld4s(S + L::KT + ty * TX + 4 * tx);
            F4 mu = ld4s(S + L::P + (ty + AH) * AW + 4 * tx + AH);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                mu.v[i] -= kd.v[i] * (d1.v[i] + d2.v[i] + hz.v[i]);
            st_own(A.ap_out + o, mu, nv);
        }
        __syncthreads();
        if (tid == 0 && it + ANS < niter) {
            fence_proxy_async_smem();
            issue(it + ANS);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            hq[j] = hq[j + 1];
            gq[j] = gq[j + 1];
        }
    }
}

template <bool kRho, bool kLocal, bool kStag>
__global__ void __launch_bounds__(NTHREADS, 2)
    adj_fused_kernel(const __grid_constant__ CUtensorMap mP, const __grid_constant__ CUtensorMap mPq,
                     const __grid_constant__ CUtensorMap mVX, const __grid_constant__ CUtensorMap mVY,
                     const __grid_constant__ CUtensorMap mVZ, const __grid_constant__ CUtensorMap mK,
                     const FusedArgs A)
{
    static_assert(TX == 32 && TY == 32 && NTHREADS == 256, "thread mapping assumes 32x32 tiles and 256 threads");
    extern __shared__ __align__(1024) float sm[];
    const Geom &G = A.g;
    const int x0 = (blockIdx.x % A.tiles_x) * TX, y0 = (blockIdx.x / A.tiles_x) * TY;
    int z0, z1;
    adj_chunk_range(A, blockIdx.y, &z0, &z1);
    const bool interior = x0 - AH >= G.lo[0] && x0 + TX + AH <= G.nx - G.hi[0] && y0 - AH >= G.lo[1] &&
                          y0 + TY + AH <= G.ny - G.hi[1] && z0 - 8 >= G.lo[2] && z1 + 8 <= G.nz - G.hi[2];
    if (interior)
        adj_body<false, kRho, false, kStag>(mP, mPq, mVX, mVY, mVZ, mK, A, z0, z1, sm);
    else
        adj_body<true, kRho, kLocal, kStag>(mP, mPq, mVX, mVY, mVZ, mK, A, z0, z1, sm);
}

}  // namespace

// One adjoint step with the fused kernel: reads the current sets of mu,
// lam_v and the memory variables, writes the other sets and flips both.
cudaError_t adjoint_step_fused(fdtd_ctx *c, const float *s_tape)
{
    static bool attr_done = false;
    if (!attr_done) {
        const void *kern[5] = {(const void *)adj_fused_kernel<false, false, false>,
                               (const void *)adj_fused_kernel<true, false, false>,
                               (const void *)adj_fused_kernel<false, true, false>,
                               (const void *)adj_fused_kernel<true, true, false>,
                               (const void *)adj_fused_kernel<false, false, true>};
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < 5 && e == cudaSuccess; ++k)
            e = cudaFuncSetAttribute(kern[k], cudaFuncAttributeMaxDynamicSharedMemorySize, FusedLayout::BYTES);
        if (e != cudaSuccess)
            return e;
        attr_done = true;
    }
    FusedArgs a;
    a.g = c->g;
    a.tiles_x = c->tiles_x;
    // z-chunks: on large grids (where the forward step has end chunks) the
    // end chunks reach 8 planes past the z slabs (the reach of lam_h_z) and
    // the middle is cut into chunks of about azchunk_target planes
    a.zmid0 = 0;
    a.zmid1 = c->g.nz;
    a.zchunk = c->zchunk;
    if (c->zmid0 > 0 || c->zmid1 < c->g.nz) {
        const int e1 = c->g.lo[2] + 8, e2 = c->g.nz - c->g.hi[2] - 8;
        const int target = c->azchunk_target;
        if (e2 - e1 >= target) {
            const int km = (e2 - e1 + target - 1) / target;
            a.zmid0 = e1;
            a.zmid1 = e2;
            a.zchunk = (e2 - e1 + km - 1) / km;
        }
    }
    a.kdt = c->kdt;
    const int s = c->aset;
    a.ap_in = c->apb[s];
    a.ap_out = c->apb[s ^ 1];
    const int nmax = max(c->g.nx, max(c->g.ny, c->g.nz));
    for (int d = 0; d < 3; ++d) {
        a.av_in[d] = c->avb[d][s];
        a.av_out[d] = c->avb[d][s ^ 1];
        a.apsiv_in[d] = c->apsiv[d][c->acur];
        a.apsiv_out[d] = c->apsiv[d][c->acur ^ 1];
        a.apsip_in[d] = c->apsip[d][c->acur];
        a.apsip_out[d] = c->apsip[d][c->acur ^ 1];
        a.cb[d] = c->coef + (d * 3 + 0) * nmax;
        a.ca[d] = c->coef + (d * 3 + 1) * nmax;
        a.ck[d] = c->coef + (d * 3 + 2) * nmax;
        const int hv = c->staggered ? 9 : 0;   // half-node tables follow the node tables
        a.cbv[d] = c->coef + (hv + d * 3 + 0) * nmax;
        a.cav[d] = c->coef + (hv + d * 3 + 1) * nmax;
        a.ckv[d] = c->coef + (hv + d * 3 + 2) * nmax;
    }
    for (int l = 0; l < 4; ++l)
        a.c[l] = (float)((c->staggered ? kStagWeights[l] : kWeights[l]) / c->d.h);
    a.dtr = (float)(c->d.dt * c->vscale);
    a.dt_over_vs = (float)(c->d.dt / c->vscale);
    for (int d = 0; d < 3; ++d)
        a.kr[d] = (float)c->kr[d];
    a.nbr = c->var_rho ? c->nbr : nullptr;
    for (int d = 0; d < 3; ++d) {
        a.lb[d] = c->cpml_local_set ? c->lcoef[d][0] : nullptr;
        a.la[d] = c->cpml_local_set ? c->lcoef[d][1] : nullptr;
    }
    a.s_tape = s_tape;
    a.gradK = c->gradK;
    a.err = c->err;
    dim3 grid(c->tiles_x * c->tiles_y, adj_chunks(a), c->d.nshots);
    const CUtensorMap *m = c->amaps[s];
    const bool loc = a.lb[0] != nullptr;
    if (c->staggered)   // constant density and the 1D grading (the API enforces both)
        adj_fused_kernel<false, false, true><<<grid, NTHREADS, FusedLayout::BYTES, c->stream>>>(
            m[0], m[1], m[2], m[3], m[4], c->mapK, a);
    else if (a.nbr && loc)
        adj_fused_kernel<true, true, false><<<grid, NTHREADS, FusedLayout::BYTES, c->stream>>>(m[0], m[1], m[2], m[3], m[4],
                                                                                        c->mapK, a);
    else if (a.nbr)
        adj_fused_kernel<true, false, false><<<grid, NTHREADS, FusedLayout::BYTES, c->stream>>>(m[0], m[1], m[2], m[3],
                                                                                         m[4], c->mapK, a);
    else if (loc)
        adj_fused_kernel<false, true, false><<<grid, NTHREADS, FusedLayout::BYTES, c->stream>>>(m[0], m[1], m[2], m[3],
                                                                                         m[4], c->mapK, a);
    else
        adj_fused_kernel<false, false, false><<<grid, NTHREADS, FusedLayout::BYTES, c->stream>>>(m[0], m[1], m[2], m[3],
                                                                                          m[4], c->mapK, a);
    const cudaError_t e = cudaGetLastError();
    c->aset ^= 1;
    c->ap = c->apb[c->aset];
    for (int d = 0; d < 3; ++d)
        c->av[d] = c->avb[d][c->aset];
    c->acur ^= 1;
    return e;
}

}  // namespace fdtd

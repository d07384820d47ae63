// Fused forward time step of the radius-4 acoustic FDTD with CPML
// (paper Sec. 3.1 leapfrog and Sec. 3.2 stretched derivative + memory
// variable), source injection and receiver sampling: one kernel per step.
//
// Data flow per CTA (tile TX x TY in x, y; a z range [z0, z1) marched plane by
// plane).  Iteration t produces:
//   v'_z at plane t+4 for the tile   (D_z p from a 9-plane register queue)
//   v'_x at plane t, tile + 4-node x halo, v'_y at plane t, tile + 4-node y
//   halo                            (D_x, D_y p from the TMA-staged plane t)
//   p'   at plane t for the tile    (D_x v'_x, D_y v'_y from shared memory,
//                                    D_z v'_z from a 9-plane register queue)
// The halo velocities are recomputed (not stored) so that one pass over HBM
// reads p, v, K once and writes p, v once (36 B per node for FP32).
// The inputs of plane t arrive through a 3-deep TMA/mbarrier pipeline; TMA
// out-of-bounds fill supplies the zero values beyond the grid.
#include "fdtd_internal.cuh"

namespace fdtd {

template <typename T>
struct StageLayout {
    static constexpr int PW = TX + 16;   // p plane with 8-node x halo
    static constexpr int PH = TY + 16;   // and 8-node y halo
    static constexpr int VXW = TX + 16;  // v_x rows with 8-node x halo (TMA-aligned for 16-bit)
    static constexpr int VYH = TY + 8;   // v_y with 4-node y halo
    static constexpr int P_BYTES = PH * PW * (int)sizeof(T);
    static constexpr int PQ_BYTES = TY * TX * (int)sizeof(T);
    static constexpr int VX_BYTES = TY * VXW * (int)sizeof(T);
    static constexpr int VY_BYTES = VYH * TX * (int)sizeof(T);
    static constexpr int VZ_BYTES = TY * TX * (int)sizeof(T);
    static constexpr int K_BYTES = TY * TX * 4;
    static constexpr int OFF_P = 0;
    static constexpr int OFF_PQ = OFF_P + P_BYTES;
    static constexpr int OFF_VX = OFF_PQ + PQ_BYTES;
    static constexpr int OFF_VY = OFF_VX + VX_BYTES;
    static constexpr int OFF_VZ = OFF_VY + VY_BYTES;
    static constexpr int OFF_K = OFF_VZ + VZ_BYTES;
    static constexpr int BYTES = OFF_K + K_BYTES;
    static_assert(OFF_PQ % 128 == 0 && OFF_VX % 128 == 0 && OFF_VY % 128 == 0 && OFF_VZ % 128 == 0 &&
                      OFF_K % 128 == 0 && BYTES % 128 == 0,
                  "TMA destinations must stay 128-byte aligned");
    static constexpr int SVX_FLOATS = TY * (TX + 8);   // v'_x, origin x0 - 4
    static constexpr int SVY_FLOATS = (TY + 8) * TX;   // v'_y, origin y0 - 4
    static constexpr int SMEM = NSTAGE * BYTES + 4 * (SVX_FLOATS + SVY_FLOATS) + 8 * NSTAGE;
};

__device__ __forceinline__ F4 f4zero() { return F4{{0.f, 0.f, 0.f, 0.f}}; }

// centred radius-4 derivative of 4 consecutive outputs from the 12 values at
// offsets -4..7 (a, b, c hold offsets -4..-1, 0..3, 4..7)
__device__ __forceinline__ F4 dx4(const F4 &a, const F4 &b, const F4 &c, const float *cw)
{
    float f[12] = {a.v[0], a.v[1], a.v[2], a.v[3], b.v[0], b.v[1], b.v[2], b.v[3], c.v[0], c.v[1], c.v[2], c.v[3]};
    F4 r;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        r.v[i] = cw[0] * (f[i + 5] - f[i + 3]) + cw[1] * (f[i + 6] - f[i + 2]) + cw[2] * (f[i + 7] - f[i + 1]) +
                 cw[3] * (f[i + 8] - f[i]);
    return r;
}

// centred derivative from 8 neighbours: m[l-1] = f(-l), p[l-1] = f(+l)
__device__ __forceinline__ F4 dn4(const F4 *m, const F4 *p, const float *cw)
{
    F4 r;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        r.v[i] = cw[0] * (p[0].v[i] - m[0].v[i]) + cw[1] * (p[1].v[i] - m[1].v[i]) +
                 cw[2] * (p[2].v[i] - m[2].v[i]) + cw[3] * (p[3].v[i] - m[3].v[i]);
    return r;
}

template <typename T>
__device__ __forceinline__ F4 lds4(const unsigned char *base, int elem)
{
    return Io<T>::ld4(reinterpret_cast<const T *>(base) + elem);
}

__device__ __forceinline__ F4 lds4f(const float *p)
{
    float4 q = *reinterpret_cast<const float4 *>(p);
    return F4{{q.x, q.y, q.z, q.w}};
}

__device__ __forceinline__ void sts4f(float *p, const F4 &v)
{
    *reinterpret_cast<float4 *>(p) = make_float4(v.v[0], v.v[1], v.v[2], v.v[3]);
}

// x-direction CPML on 4 consecutive nodes starting at gx (row y, plane z):
// psi <- b psi + a g ; g <- kinv g + psi.  Reads psi from `pin`, writes to
// `pout` when write is set (pout may equal pin).  Optionally tapes (g, psi_old).
template <typename T>
__device__ __forceinline__ void cpml_x(const Geom &G, const StepArgs &A, F4 &gv, const T *pin, T *pout,
                                       int z, int y, int gx, bool write, float *tape, int tape_off)
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int x = gx + i;
        if (x < G.nx && in_slab(x, G.nx, G.lo[0], G.hi[0])) {
            long long idx = ((long long)z * G.ny + y) * G.w[0] + slab_coord(x, G.nx, G.lo[0], G.hi[0]);
            float ps = Io<T>::ld1(pin + idx);
            float b = __ldg(A.cb[0] + x), a = __ldg(A.ca[0] + x), k = __ldg(A.ck[0] + x);
            float pn = b * ps + a * gv.v[i];
            if (tape) {
                tape[idx * 4 + tape_off] = gv.v[i];
                tape[idx * 4 + tape_off + 1] = ps;
            }
            gv.v[i] = k * gv.v[i] + pn;
            if (write)
                Io<T>::st1(pout + idx, pn);
        }
    }
}

// y- or z-direction CPML: the 4 nodes share one profile value and are
// contiguous in the memory-variable array.
template <typename T>
__device__ __forceinline__ void cpml_yz(F4 &gv, const T *pin, T *pout, long long idx, float b, float a, float k,
                                        bool write, int nvalid, float *tape, int tape_off)
{
    F4 ps = Io<T>::ld4(pin + idx);
    F4 pn;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        pn.v[i] = b * ps.v[i] + a * gv.v[i];
        if (tape && i < nvalid) {
            tape[(idx + i) * 4 + tape_off] = gv.v[i];
            tape[(idx + i) * 4 + tape_off + 1] = ps.v[i];
        }
        gv.v[i] = k * gv.v[i] + pn.v[i];
    }
    if (write)
        Io<T>::st4(pout + idx, pn);
}

template <typename T>
__global__ void __launch_bounds__(NTHREADS, 2)
    fdtd_step_kernel(const __grid_constant__ CUtensorMap mP, const __grid_constant__ CUtensorMap mPq,
                     const __grid_constant__ CUtensorMap mVX, const __grid_constant__ CUtensorMap mVY,
                     const __grid_constant__ CUtensorMap mVZ, const __grid_constant__ CUtensorMap mK,
                     const StepArgs A)
{
    using L = StageLayout<T>;
    extern __shared__ __align__(1024) unsigned char smem[];
    float *svx = reinterpret_cast<float *>(smem + NSTAGE * L::BYTES);
    float *svy = svx + L::SVX_FLOATS;
    uint64_t *bar = reinterpret_cast<uint64_t *>(svy + L::SVY_FLOATS);

    const Geom &G = A.g;
    const int tid = threadIdx.x;
    const int tx = tid % (TX / 4), ty = tid / (TX / 4);
    const int tile = blockIdx.x;
    const int x0 = (tile % A.tiles_x) * TX, y0 = (tile / A.tiles_x) * TY;
    const int z0 = blockIdx.y * A.zchunk;
    const int z1 = min(G.nz, z0 + A.zchunk);
    const int shot = blockIdx.z;
    const int gx = x0 + 4 * tx, gy = y0 + ty;
    const int niter = z1 - z0 + 8;
    const float cw[4] = {A.c[0], A.c[1], A.c[2], A.c[3]};

    const long long fofs = (long long)shot * G.vol;
    const T *p_in = reinterpret_cast<const T *>(A.p_in) + fofs;
    T *p_out = reinterpret_cast<T *>(A.p_out) + fofs;
    T *v_out[3];
    const T *psiv_in[3];
    T *psiv_out[3], *psip[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        v_out[d] = reinterpret_cast<T *>(A.v_out[d]) + fofs;
        psiv_in[d] = reinterpret_cast<const T *>(A.psiv_in[d]) + (long long)shot * G.slab[d];
        psiv_out[d] = reinterpret_cast<T *>(A.psiv_out[d]) + (long long)shot * G.slab[d];
        psip[d] = reinterpret_cast<T *>(A.psip[d]) + (long long)shot * G.slab[d];
    }
    float *stape[3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
        stape[d] = A.slab_tape[d] ? A.slab_tape[d] + (long long)shot * G.slab[d] * 4 : nullptr;

    // which of this thread's 4 own nodes lie inside the grid
    bool own_ok[4];
    int nvalid = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        own_ok[i] = (gx + i < G.nx) && (gy < G.ny);
        nvalid += own_ok[i] ? 1 : 0;
    }
    const bool row_ok = gy < G.ny && gx < G.nxp;

    // source of this shot
    const int sz = A.src ? A.src[3 * shot] : -1, sy = A.src ? A.src[3 * shot + 1] : -1,
              sx = A.src ? A.src[3 * shot + 2] : -1;
    const float wsrc = (A.src && A.t < A.nt_w) ? A.wavelet[(long long)shot * A.nt_w + A.t] : 0.f;
    // receivers of this tile (sorted by z)
    int rc = 0, r1 = 0;
    const bool rec_on = A.traces != nullptr && A.nrec > 0 && A.t < A.nt_max;
    if (rec_on) {
        rc = A.rec_off[tile];
        r1 = A.rec_off[tile + 1];
    }

    if (tid == 0) {
        prefetch_tmap(&mP);
        prefetch_tmap(&mPq);
        prefetch_tmap(&mVX);
        prefetch_tmap(&mVY);
        prefetch_tmap(&mVZ);
        prefetch_tmap(&mK);
        for (int s = 0; s < NSTAGE; ++s)
            mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // Issue the loads of iteration `it` into its stage (thread 0 only).
    auto issue = [&](int it) {
        const int t = z0 - 8 + it;
        unsigned char *S = smem + (it % NSTAGE) * L::BYTES;
        uint64_t *b = &bar[it % NSTAGE];
        uint32_t bytes = 0;
        const bool q_on = (t + 8 >= 0) && (t + 8 < G.nz);
        const bool vz_on = (t + 4 >= 0) && (t + 4 < G.nz);
        const bool main_on = t >= z0;
        bytes += q_on ? L::PQ_BYTES : 0;
        bytes += vz_on ? L::VZ_BYTES : 0;
        bytes += main_on ? (L::P_BYTES + L::VX_BYTES + L::VY_BYTES + L::K_BYTES) : 0;
        mbar_arrive_expect_tx(b, bytes);
        if (q_on)
            tma_load_4d(S + L::OFF_PQ, &mPq, b, x0, y0, t + 8, shot);
        if (vz_on)
            tma_load_4d(S + L::OFF_VZ, &mVZ, b, x0, y0, t + 4, shot);
        if (main_on) {
            tma_load_4d(S + L::OFF_P, &mP, b, x0 - 8, y0 - 8, t, shot);
            tma_load_4d(S + L::OFF_VX, &mVX, b, x0 - 8, y0, t, shot);
            tma_load_4d(S + L::OFF_VY, &mVY, b, x0, y0 - 4, t, shot);
            tma_load_3d(S + L::OFF_K, &mK, b, x0, y0, t);
        }
    };
    if (tid == 0)
        for (int i = 0; i < NSTAGE && i < niter; ++i)
            issue(i);

    // register queues: pq[k] = p(t + k), vzq[k] = v'_z(t - 4 + k)
    F4 pq[9], vzq[9];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int z = z0 - 8 + k;
        pq[k] = f4zero();
        if (z >= 0 && row_ok) {
            F4 q = Io<T>::ldg4(p_in + (long long)z * G.plane + (long long)gy * G.nxp + gx);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                pq[k].v[i] = own_ok[i] ? q.v[i] : 0.f;
        }
        vzq[k] = f4zero();
    }
    pq[8] = f4zero();
    vzq[8] = f4zero();

    for (int it = 0; it < niter; ++it) {
        const int t = z0 - 8 + it;
        const unsigned char *S = smem + (it % NSTAGE) * L::BYTES;
        const bool ok = mbar_wait_bounded(&bar[it % NSTAGE], (it / NSTAGE) & 1, WAIT_LIMIT);

        // ---- p(t + 8) into the queue
        pq[8] = f4zero();
        if (ok && t + 8 < G.nz) {
            F4 q = lds4<T>(S + L::OFF_PQ, ty * TX + 4 * tx);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                pq[8].v[i] = own_ok[i] ? q.v[i] : 0.f;
        }

        // ---- v'_z at plane t + 4 (velocity half step, z component)
        const int zv = t + 4;
        F4 vzn = f4zero();
        if (ok && zv >= 0 && zv < G.nz) {
            F4 gz;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                gz.v[i] = cw[0] * (pq[5].v[i] - pq[3].v[i]) + cw[1] * (pq[6].v[i] - pq[2].v[i]) +
                          cw[2] * (pq[7].v[i] - pq[1].v[i]) + cw[3] * (pq[8].v[i] - pq[0].v[i]);
            const bool owned = zv >= z0 && zv < z1;
            if (row_ok && in_slab(zv, G.nz, G.lo[2], G.hi[2])) {
                const long long idx = slab_index(G, 2, zv, gy, gx);
                cpml_yz<T>(gz, psiv_in[2], psiv_out[2], idx, __ldg(A.cb[2] + zv), __ldg(A.ca[2] + zv),
                           __ldg(A.ck[2] + zv), owned, nvalid, owned ? stape[2] : nullptr, 0);
            }
            F4 vo = lds4<T>(S + L::OFF_VZ, ty * TX + 4 * tx);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                vzn.v[i] = own_ok[i] ? vo.v[i] - A.dtr * gz.v[i] : 0.f;
            if (owned && row_ok)
                Io<T>::st4(v_out[2] + (long long)zv * G.plane + (long long)gy * G.nxp + gx, vzn);
        }
        vzq[8] = vzn;

        const bool active = t >= z0;
        if (ok && active) {
            const unsigned char *Sp = S + L::OFF_P;   // p plane, origin (x0 - 8, y0 - 8)
            // ---- v'_x, own nodes
            {
                const int lrow = (ty + 8) * L::PW, lx = 4 * tx + 8;
                F4 g = dx4(lds4<T>(Sp, lrow + lx - 4), lds4<T>(Sp, lrow + lx), lds4<T>(Sp, lrow + lx + 4), cw);
                if (gy < G.ny && (gx < G.lo[0] || gx + 3 >= G.nx - G.hi[0]))
                    cpml_x<T>(G, A, g, psiv_in[0], psiv_out[0], t, gy, gx, true, stape[0], 0);
                F4 vo = lds4<T>(S + L::OFF_VX, ty * L::VXW + 4 * tx + 8);
                F4 vn;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    vn.v[i] = own_ok[i] ? vo.v[i] - A.dtr * g.v[i] : 0.f;
                if (row_ok)
                    Io<T>::st4(v_out[0] + (long long)t * G.plane + (long long)gy * G.nxp + gx, vn);
                sts4f(svx + ty * (TX + 8) + 4 * tx + 4, vn);
            }
            // ---- v'_x, 4-node x halo on both sides (recomputed, not stored)
            if (tid < 2 * TY) {
                const int r = tid >> 1, side = tid & 1;
                const int hx = side ? x0 + TX : x0 - 4;
                const int hy = y0 + r;
                const int lrow = (r + 8) * L::PW, lx = hx - x0 + 8;
                F4 g = dx4(lds4<T>(Sp, lrow + lx - 4), lds4<T>(Sp, lrow + lx), lds4<T>(Sp, lrow + lx + 4), cw);
                if (hy < G.ny && hx >= 0 && hx < G.nx)
                    cpml_x<T>(G, A, g, psiv_in[0], psiv_out[0], t, hy, hx, false, nullptr, 0);
                F4 vo = lds4<T>(S + L::OFF_VX, r * L::VXW + lx);
                F4 vn;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const bool in = hy < G.ny && hx + i >= 0 && hx + i < G.nx;
                    vn.v[i] = in ? vo.v[i] - A.dtr * g.v[i] : 0.f;
                }
                sts4f(svx + r * (TX + 8) + (hx - x0 + 4), vn);
            }
            // ---- v'_y, own nodes
            {
                const int lx = 4 * tx + 8, ly = ty + 8;
                F4 m[4], p[4];
#pragma unroll
                for (int l = 1; l <= 4; ++l) {
                    m[l - 1] = lds4<T>(Sp, (ly - l) * L::PW + lx);
                    p[l - 1] = lds4<T>(Sp, (ly + l) * L::PW + lx);
                }
                F4 g = dn4(m, p, cw);
                if (row_ok && in_slab(gy, G.ny, G.lo[1], G.hi[1])) {
                    const long long idx = slab_index(G, 1, t, gy, gx);
                    cpml_yz<T>(g, psiv_in[1], psiv_out[1], idx, __ldg(A.cb[1] + gy), __ldg(A.ca[1] + gy),
                               __ldg(A.ck[1] + gy), true, nvalid, stape[1], 0);
                }
                F4 vo = lds4<T>(S + L::OFF_VY, (ty + 4) * TX + 4 * tx);
                F4 vn;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    vn.v[i] = own_ok[i] ? vo.v[i] - A.dtr * g.v[i] : 0.f;
                if (row_ok)
                    Io<T>::st4(v_out[1] + (long long)t * G.plane + (long long)gy * G.nxp + gx, vn);
                sts4f(svy + (ty + 4) * TX + 4 * tx, vn);
            }
            // ---- v'_y, 4-row y halo above and below (recomputed, not stored)
            for (int hsk = tid; hsk < 8 * (TX / 4); hsk += NTHREADS) {
                const int r = hsk / (TX / 4), c = hsk % (TX / 4);
                const int hy = r < 4 ? y0 - 4 + r : y0 + TY + (r - 4);
                const int hx = x0 + 4 * c;
                const int ly = hy - y0 + 8, lx = 4 * c + 8;
                F4 m[4], p[4];
#pragma unroll
                for (int l = 1; l <= 4; ++l) {
                    m[l - 1] = lds4<T>(Sp, (ly - l) * L::PW + lx);
                    p[l - 1] = lds4<T>(Sp, (ly + l) * L::PW + lx);
                }
                F4 g = dn4(m, p, cw);
                const bool yin = hy >= 0 && hy < G.ny;
                if (yin && hx < G.nxp && in_slab(hy, G.ny, G.lo[1], G.hi[1])) {
                    const long long idx = slab_index(G, 1, t, hy, hx);
                    cpml_yz<T>(g, psiv_in[1], psiv_out[1], idx, __ldg(A.cb[1] + hy), __ldg(A.ca[1] + hy),
                               __ldg(A.ck[1] + hy), false, 0, nullptr, 0);
                }
                F4 vo = lds4<T>(S + L::OFF_VY, (hy - y0 + 4) * TX + 4 * c);
                F4 vn;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    vn.v[i] = (yin && hx + i < G.nx) ? vo.v[i] - A.dtr * g.v[i] : 0.f;
                sts4f(svy + (hy - y0 + 4) * TX + 4 * c, vn);
            }
        }

        // all v' of plane t are in shared memory; abort together on a timeout
        if (__syncthreads_or(ok ? 0 : 1)) {
            if (tid == 0) {
                atomicOr(A.err, ERR_TIMEOUT);
                for (int j = it; j < niter && j < it + NSTAGE; ++j)
                    mbar_wait_bounded(&bar[j % NSTAGE], (j / NSTAGE) & 1, WAIT_LIMIT_DRAIN);
            }
            return;
        }

        if (active) {
            // ---- pressure step at plane t
            F4 hx4 = dx4(lds4f(svx + ty * (TX + 8) + 4 * tx), lds4f(svx + ty * (TX + 8) + 4 * tx + 4),
                         lds4f(svx + ty * (TX + 8) + 4 * tx + 8), cw);
            F4 hy4;
            {
                F4 m[4], p[4];
#pragma unroll
                for (int l = 1; l <= 4; ++l) {
                    m[l - 1] = lds4f(svy + (ty + 4 - l) * TX + 4 * tx);
                    p[l - 1] = lds4f(svy + (ty + 4 + l) * TX + 4 * tx);
                }
                hy4 = dn4(m, p, cw);
            }
            F4 hz4;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                hz4.v[i] = cw[0] * (vzq[5].v[i] - vzq[3].v[i]) + cw[1] * (vzq[6].v[i] - vzq[2].v[i]) +
                           cw[2] * (vzq[7].v[i] - vzq[1].v[i]) + cw[3] * (vzq[8].v[i] - vzq[0].v[i]);
            if (gy < G.ny && (gx < G.lo[0] || gx + 3 >= G.nx - G.hi[0]))
                cpml_x<T>(G, A, hx4, psip[0], psip[0], t, gy, gx, true, stape[0], 2);
            if (row_ok && in_slab(gy, G.ny, G.lo[1], G.hi[1])) {
                const long long idx = slab_index(G, 1, t, gy, gx);
                cpml_yz<T>(hy4, psip[1], psip[1], idx, __ldg(A.cb[1] + gy), __ldg(A.ca[1] + gy),
                           __ldg(A.ck[1] + gy), true, nvalid, stape[1], 2);
            }
            if (row_ok && in_slab(t, G.nz, G.lo[2], G.hi[2])) {
                const long long idx = slab_index(G, 2, t, gy, gx);
                cpml_yz<T>(hz4, psip[2], psip[2], idx, __ldg(A.cb[2] + t), __ldg(A.ca[2] + t),
                           __ldg(A.ck[2] + t), true, nvalid, stape[2], 2);
            }
            const F4 kd = lds4f(reinterpret_cast<const float *>(S + L::OFF_K) + ty * TX + 4 * tx);
            F4 pn, sb;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                sb.v[i] = hx4.v[i] + hy4.v[i] + hz4.v[i];
                pn.v[i] = own_ok[i] ? pq[0].v[i] - kd.v[i] * sb.v[i] : 0.f;
            }
            if (t == sz && gy == sy && sx >= gx && sx < gx + 4)
                pn.v[sx - gx] += wsrc;
            if (row_ok) {
                const long long o = (long long)t * G.plane + (long long)gy * G.nxp + gx;
                Io<T>::st4(p_out + o, pn);
                if (A.s_tape)
                    sts4f(A.s_tape + fofs + o, sb);
            }
            if (rec_on) {
                while (rc < r1 && A.rec[rc].x < t)
                    ++rc;
                for (int r = rc; r < r1; ++r) {
                    const int4 q = A.rec[r];
                    if (q.x != t)
                        break;
                    if (q.y == gy && q.z >= gx && q.z < gx + 4) {
                        // re-read through the storage type so traces equal the stored state
                        T tmp = T(pn.v[q.z - gx]);
                        A.traces[((long long)shot * A.nt_max + A.t) * A.nrec + q.w] = Io<T>::ld1(&tmp);
                    }
                }
            }
        }
        __syncthreads();
        if (tid == 0 && it + NSTAGE < niter) {
            fence_proxy_async_smem();
            issue(it + NSTAGE);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            pq[k] = pq[k + 1];
            vzq[k] = vzq[k + 1];
        }
    }
}

template <typename T>
static cudaError_t launch_step_t(const fdtd_ctx *c, const StepArgs &a, int set)
{
    using L = StageLayout<T>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(fdtd_step_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             L::SMEM);
        if (e != cudaSuccess)
            return e;
        attr_done = true;
    }
    dim3 grid(c->tiles_x * c->tiles_y, c->nzchunks, c->d.nshots);
    fdtd_step_kernel<T><<<grid, NTHREADS, L::SMEM, c->stream>>>(c->maps[set][0], c->maps[set][1], c->maps[set][2],
                                                                 c->maps[set][3], c->maps[set][4], c->mapK, a);
    return cudaGetLastError();
}

cudaError_t launch_step(const fdtd_ctx *c, const StepArgs &a, int set)
{
    switch (c->d.storage) {
    case FDTD_F16:
        return launch_step_t<__half>(c, a, set);
    case FDTD_BF16:
        return launch_step_t<__nv_bfloat16>(c, a, set);
    default:
        return launch_step_t<float>(c, a, set);
    }
}

int step_smem_bytes(int storage)
{
    switch (storage) {
    case FDTD_F16:
        return StageLayout<__half>::SMEM;
    case FDTD_BF16:
        return StageLayout<__nv_bfloat16>::SMEM;
    default:
        return StageLayout<float>::SMEM;
    }
}

int step_occupancy(int storage, int *blocks)
{
    cudaError_t e;
    switch (storage) {
    case FDTD_F16:
        cudaFuncSetAttribute(fdtd_step_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             StageLayout<__half>::SMEM);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fdtd_step_kernel<__half>, NTHREADS,
                                                          StageLayout<__half>::SMEM);
        break;
    case FDTD_BF16:
        cudaFuncSetAttribute(fdtd_step_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             StageLayout<__nv_bfloat16>::SMEM);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fdtd_step_kernel<__nv_bfloat16>, NTHREADS,
                                                          StageLayout<__nv_bfloat16>::SMEM);
        break;
    default:
        cudaFuncSetAttribute(fdtd_step_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             StageLayout<float>::SMEM);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fdtd_step_kernel<float>, NTHREADS,
                                                          StageLayout<float>::SMEM);
    }
    return e == cudaSuccess ? 0 : -1;
}

}  // namespace fdtd

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
//
// Arithmetic is FP32 in registers, packed two nodes per instruction
// (FFMA2/FMUL2/FADD2).  In the CPML slabs the memory variables of the next
// plane are prefetched into L2 one plane ahead; the CPML update is the same
// vector formula everywhere, since the coefficient tables hold b = a = 0,
// 1/kappa = 1 outside the slabs.
#include "fdtd_internal.cuh"

namespace fdtd {

// 2 CTAs of 256 threads per SM (128 registers per thread)
constexpr int kMinBlocks = 2;

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
    static constexpr int SVXW = TX + 8;                // v'_x row, origin x0 - 4
    static constexpr int SVX_FLOATS = TY * SVXW;
    static constexpr int SVY_FLOATS = (TY + 8) * TX;   // v'_y, origin y0 - 4
    static constexpr int SMEM = NSTAGE * BYTES + 4 * (SVX_FLOATS + SVY_FLOATS) + 8 * NSTAGE;
};

// four consecutive x nodes as two packed pairs
struct V4 {
    float2 a, b;
};

__device__ __forceinline__ V4 v4zero() { return V4{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
__device__ __forceinline__ V4 to_v4(const F4 &f) { return V4{make_float2(f.v[0], f.v[1]), make_float2(f.v[2], f.v[3])}; }
__device__ __forceinline__ F4 to_f4(const V4 &v) { return F4{{v.a.x, v.a.y, v.b.x, v.b.y}}; }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ V4 fma4(float2 s, const V4 &x, const V4 &y) { return V4{fma2(s, x.a, y.a), fma2(s, x.b, y.b)}; }
__device__ __forceinline__ V4 mul4(const V4 &x, const V4 &y) { return V4{mul2(x.a, y.a), mul2(x.b, y.b)}; }
__device__ __forceinline__ V4 add4(const V4 &x, const V4 &y) { return V4{add2(x.a, y.a), add2(x.b, y.b)}; }

template <typename T>
__device__ __forceinline__ V4 lds(const unsigned char *base, int elem)
{
    return to_v4(Io<T>::ld4(reinterpret_cast<const T *>(base) + elem));
}

__device__ __forceinline__ V4 ldsf(const float *p)
{
    float4 q = *reinterpret_cast<const float4 *>(p);
    return V4{make_float2(q.x, q.y), make_float2(q.z, q.w)};
}

__device__ __forceinline__ void stsf(float *p, const V4 &v)
{
    *reinterpret_cast<float4 *>(p) = make_float4(v.a.x, v.a.y, v.b.x, v.b.y);
}

// Coefficients a_l / h as packed pairs: cp = (c, c), cn = (-c, -c).
struct Coef {
    float2 cp[4], cn[4];
};

// centred derivative from aligned neighbours: m[l-1] = f(-l), p[l-1] = f(+l).
// kSplit: two independent chains (l = 1, 2 and l = 3, 4) and their sum, which
// shortens the dependency chain; the 16-bit forms, whose instruction stream
// dominates their time, use it (FP32 keeps the single chain, which measured
// faster there)
template <bool kSplit = false>
__device__ __forceinline__ V4 dnb(const V4 *m, const V4 *p, const Coef &C)
{
    if (kSplit) {
        V4 r, s;
        r.a = mul2(C.cp[0], p[0].a);
        r.b = mul2(C.cp[0], p[0].b);
        s.a = mul2(C.cp[2], p[2].a);
        s.b = mul2(C.cp[2], p[2].b);
        r.a = fma2(C.cn[0], m[0].a, r.a);
        r.b = fma2(C.cn[0], m[0].b, r.b);
        s.a = fma2(C.cn[2], m[2].a, s.a);
        s.b = fma2(C.cn[2], m[2].b, s.b);
        r.a = fma2(C.cp[1], p[1].a, r.a);
        r.b = fma2(C.cp[1], p[1].b, r.b);
        s.a = fma2(C.cp[3], p[3].a, s.a);
        s.b = fma2(C.cp[3], p[3].b, s.b);
        r.a = fma2(C.cn[1], m[1].a, r.a);
        r.b = fma2(C.cn[1], m[1].b, r.b);
        s.a = fma2(C.cn[3], m[3].a, s.a);
        s.b = fma2(C.cn[3], m[3].b, s.b);
        return V4{add2(r.a, s.a), add2(r.b, s.b)};
    }
    V4 r;
    r.a = mul2(C.cp[0], p[0].a);
    r.b = mul2(C.cp[0], p[0].b);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        if (l > 0) {
            r.a = fma2(C.cp[l], p[l].a, r.a);
            r.b = fma2(C.cp[l], p[l].b, r.b);
        }
        r.a = fma2(C.cn[l], m[l].a, r.a);
        r.b = fma2(C.cn[l], m[l].b, r.b);
    }
    return r;
}

// x derivative of 4 consecutive outputs from the 12 values at offsets -4..7
// (u, v, w hold offsets -4..-1, 0..3, 4..7).  Even offsets pair up with the
// packed layout; odd offsets use scalar FMAs on the same accumulators.
__device__ __forceinline__ V4 dx4(const V4 &u, const V4 &v, const V4 &w, const Coef &C)
{
    const float f[12] = {u.a.x, u.a.y, u.b.x, u.b.y, v.a.x, v.a.y, v.b.x, v.b.y, w.a.x, w.a.y, w.b.x, w.b.y};
    // packed pairs P[k] = (f[2k], f[2k+1])
    const float2 P0 = u.a, P1 = u.b, P2 = v.a, P3 = v.b, P4 = w.a, P5 = w.b;
    V4 r;
    // l = 2, 4 (aligned): pair (o0,o1) centred at f4,f5; pair (o2,o3) at f6,f7
    r.a = mul2(C.cp[1], P3);
    r.a = fma2(C.cn[1], P1, r.a);
    r.a = fma2(C.cp[3], P4, r.a);
    r.a = fma2(C.cn[3], P0, r.a);
    r.b = mul2(C.cp[1], P4);
    r.b = fma2(C.cn[1], P2, r.b);
    r.b = fma2(C.cp[3], P5, r.b);
    r.b = fma2(C.cn[3], P1, r.b);
    // l = 1, 3 (odd offsets), scalar
    const float c1 = C.cp[0].x, c3 = C.cp[2].x;
    r.a.x = fmaf(c1, f[5] - f[3], r.a.x);
    r.a.y = fmaf(c1, f[6] - f[4], r.a.y);
    r.b.x = fmaf(c1, f[7] - f[5], r.b.x);
    r.b.y = fmaf(c1, f[8] - f[6], r.b.y);
    r.a.x = fmaf(c3, f[7] - f[1], r.a.x);
    r.a.y = fmaf(c3, f[8] - f[2], r.a.y);
    r.b.x = fmaf(c3, f[9] - f[3], r.b.x);
    r.b.y = fmaf(c3, f[10] - f[4], r.b.y);
    return r;
}

// The same two operations on one pair of nodes, with the operation order of
// the first pair of dnb / dx4, so that a recomputed halo pair equals what the
// neighbouring tile computes for its own nodes, bit for bit.
template <bool kSplit = false>
__device__ __forceinline__ float2 dnb2(const float2 *m, const float2 *p, const Coef &C)
{
    if (kSplit) {   // the order of dnb<true>
        float2 r = mul2(C.cp[0], p[0]), s = mul2(C.cp[2], p[2]);
        r = fma2(C.cn[0], m[0], r);
        s = fma2(C.cn[2], m[2], s);
        r = fma2(C.cp[1], p[1], r);
        s = fma2(C.cp[3], p[3], s);
        r = fma2(C.cn[1], m[1], r);
        s = fma2(C.cn[3], m[3], s);
        return add2(r, s);
    }
    float2 r = mul2(C.cp[0], p[0]);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        if (l > 0)
            r = fma2(C.cp[l], p[l], r);
        r = fma2(C.cn[l], m[l], r);
    }
    return r;
}

// x derivative of the pair at offsets 4, 5 of P0..P4 (offsets 0..9)
__device__ __forceinline__ float2 dx2(float2 P0, float2 P1, float2 P2, float2 P3, float2 P4, const Coef &C)
{
    float2 r = mul2(C.cp[1], P3);
    r = fma2(C.cn[1], P1, r);
    r = fma2(C.cp[3], P4, r);
    r = fma2(C.cn[3], P0, r);
    const float c1 = C.cp[0].x, c3 = C.cp[2].x;
    r.x = fmaf(c1, P2.y - P1.y, r.x);
    r.y = fmaf(c1, P3.x - P2.x, r.y);
    r.x = fmaf(c3, P3.y - P0.y, r.x);
    r.y = fmaf(c3, P4.x - P1.x, r.y);
    return r;
}

// Staggered (Yee) form: v_d[i] lives at i + 1/2.  With c_l / h in C:
//   forward  (p -> v at i):  sum_l c_l (f[i + l] - f[i + 1 - l])
//   backward (v -> p at i):  sum_l c_l (f[i + l - 1] - f[i - l])
// For a pair of outputs one of the two terms of each l falls on an aligned
// pair (packed FMA) and the other does not (two scalar FMAs).
// Forward derivative of the pair at offsets 4, 5 of P0..P4 (offsets 0..9).
__device__ __forceinline__ float2 sdf2(float2 P0, float2 P1, float2 P2, float2 P3, float2 P4, const Coef &C)
{
    float2 r = mul2(C.cp[1], P3);       // l = 2: f(+2), f(+3)
    r = fma2(C.cp[3], P4, r);           // l = 4: f(+4), f(+5)
    r = fma2(C.cn[0], P2, r);           // l = 1: f(0), f(1)
    r = fma2(C.cn[2], P1, r);           // l = 3: f(-2), f(-1)
    const float c1 = C.cp[0].x, c3 = C.cp[2].x, m2 = C.cn[1].x, m4 = C.cn[3].x;
    r.x = fmaf(c1, P2.y, r.x);          // l = 1: f(+1)
    r.y = fmaf(c1, P3.x, r.y);
    r.x = fmaf(m2, P1.y, r.x);          // l = 2: f(-1)
    r.y = fmaf(m2, P2.x, r.y);
    r.x = fmaf(c3, P3.y, r.x);          // l = 3: f(+3)
    r.y = fmaf(c3, P4.x, r.y);
    r.x = fmaf(m4, P0.y, r.x);          // l = 4: f(-3)
    r.y = fmaf(m4, P1.x, r.y);
    return r;
}

// forward derivative of 4 outputs from offsets -4..7 (u, v, w as in dx4);
// each pair takes the operation order of sdf2, so halo pairs match
__device__ __forceinline__ V4 sdf4(const V4 &u, const V4 &v, const V4 &w, const Coef &C)
{
    return V4{sdf2(u.a, u.b, v.a, v.b, w.a, C), sdf2(u.b, v.a, v.b, w.a, w.b, C)};
}

// backward derivative of the pair at offsets 4, 5 of P0..P4 (offsets 0..9)
__device__ __forceinline__ float2 sdb2(float2 P0, float2 P1, float2 P2, float2 P3, float2 P4, const Coef &C)
{
    float2 r = mul2(C.cp[0], P2);       // l = 1: f(0), f(1)
    r = fma2(C.cp[2], P3, r);           // l = 3: f(+2), f(+3)
    r = fma2(C.cn[1], P1, r);           // l = 2: f(-2), f(-1)
    r = fma2(C.cn[3], P0, r);           // l = 4: f(-4), f(-3)
    const float c2 = C.cp[1].x, c4 = C.cp[3].x, m1 = C.cn[0].x, m3 = C.cn[2].x;
    r.x = fmaf(m1, P1.y, r.x);          // l = 1: f(-1)
    r.y = fmaf(m1, P2.x, r.y);
    r.x = fmaf(c2, P2.y, r.x);          // l = 2: f(+1)
    r.y = fmaf(c2, P3.x, r.y);
    r.x = fmaf(m3, P0.y, r.x);          // l = 3: f(-3)
    r.y = fmaf(m3, P1.x, r.y);
    r.x = fmaf(c4, P3.y, r.x);          // l = 4: f(+3)
    r.y = fmaf(c4, P4.x, r.y);
    return r;
}

__device__ __forceinline__ V4 sdb4(const V4 &u, const V4 &v, const V4 &w, const Coef &C)
{
    return V4{sdb2(u.a, u.b, v.a, v.b, w.a, C), sdb2(u.b, v.a, v.b, w.a, w.b, C)};
}

__device__ __forceinline__ void cpml2(float2 &g, float2 psi, float2 b, float2 a, float2 k)
{
    const float2 pn = fma2(b, psi, mul2(a, g));
    g = fma2(k, g, pn);
}

template <typename T>
__device__ __forceinline__ float2 lds2(const unsigned char *base, int elem)
{
    return Io<T>::ld2(reinterpret_cast<const T *>(base) + elem);
}

// One CPML update of 4 nodes: psi' = b psi + a g ; g' = kinv g + psi'.
__device__ __forceinline__ V4 cpml4(V4 &g, const V4 &psi, const V4 &b, const V4 &a, const V4 &k)
{
    V4 pn;
    pn.a = fma2(b.a, psi.a, mul2(a.a, g.a));
    pn.b = fma2(b.b, psi.b, mul2(a.b, g.b));
    g.a = fma2(k.a, g.a, pn.a);
    g.b = fma2(k.b, g.b, pn.b);
    return pn;
}

__device__ __forceinline__ V4 splat4(float s) { return V4{make_float2(s, s), make_float2(s, s)}; }

// x + s y with a per-node factor s (variable density)
__device__ __forceinline__ V4 fmav(const V4 &s, const V4 &x, const V4 &y)
{
    return V4{fma2(s.a, x.a, y.a), fma2(s.b, x.b, y.b)};
}

// -dt vscale / rho of 4 nodes (0 when the row is outside the grid)
__device__ __forceinline__ V4 ld_nbr(const float *nbr, long long o, bool ok)
{
    return ok ? to_v4(Io<float>::ldg4(nbr + o)) : v4zero();
}

template <typename T>
__device__ __forceinline__ V4 ldg_v4(const T *p) { return to_v4(Io<T>::ld4(p)); }

// per-node CPML coefficients of 4 nodes (local grading tables, read-only)
__device__ __forceinline__ V4 ldc4(const float *p) { return to_v4(Io<float>::ldg4(p)); }
__device__ __forceinline__ float2 ldc2(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }

// store of a step output, not read again within this step: L2 evict-first
template <typename T>
__device__ __forceinline__ void st_out(T *p, const F4 &v)
{
    Io<T>::st4s(p, v);
}

// tape (g, psi_old) of 4 nodes into slots [idx*4 + off, +1]
__device__ __forceinline__ void tape4(float *tape, long long idx, int off, const V4 &g, const V4 &psi)
{
    const F4 gf = to_f4(g), pf = to_f4(psi);
#pragma unroll
    for (int i = 0; i < 4; ++i)
        *reinterpret_cast<float2 *>(tape + (idx + i) * 4 + off) = make_float2(gf.v[i], pf.v[i]);
}

// Queue work of one plane.  Logical entry j of each 9-deep queue lives in
// slot j: pq[j] = p(t + j), vzq[j] = v'_z(t - 4 + j); the queues shift by one
// slot per plane.  kStag: v_z[t + 4] sits at t + 4.5 and the pressure at t
// reads v_z at t - 4 .. t + 3 (the staggered neighbour sets).
template <bool kStag, bool kSplit, typename Zvel>
__device__ __forceinline__ void zblock(V4 (&pq)[9], V4 (&vzq)[9], const V4 &pnew, const Coef &C, Zvel &&zvel,
                                       V4 &pt, V4 &hz)
{
    pq[8] = pnew;
    V4 gz;
    {
        const V4 m[4] = {pq[kStag ? 4 : 3], pq[kStag ? 3 : 2], pq[kStag ? 2 : 1], pq[kStag ? 1 : 0]};
        const V4 p[4] = {pq[5], pq[6], pq[7], pq[8]};
        gz = dnb<kSplit>(m, p, C);
    }
    pt = pq[0];
    vzq[8] = zvel(gz);
    {
        const V4 m[4] = {vzq[3], vzq[2], vzq[1], vzq[0]};
        const V4 p[4] = {vzq[kStag ? 4 : 5], vzq[kStag ? 5 : 6], vzq[kStag ? 6 : 7], vzq[kStag ? 7 : 8]};
        hz = dnb<kSplit>(m, p, C);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        pq[k] = pq[k + 1];
        vzq[k] = vzq[k + 1];
    }
}

// z range of chunk y of a launch (see StepArgs::zmid0).  The zchunk-plane
// chunks of [zmid0, zmid1) come first, the shorter end chunks last, so that
// the long chunks start in the first waves.
__host__ __device__ __forceinline__ void chunk_range(const StepArgs &A, int y, int *z0, int *z1)
{
    const int nmid = (A.zmid1 - A.zmid0 + A.zchunk - 1) / A.zchunk;
    if (y < nmid) {
        *z0 = A.zmid0 + y * A.zchunk;
        *z1 = min(A.zmid1, *z0 + A.zchunk);
    } else if (y == nmid && A.zmid0 > A.zbase) {
        *z0 = A.zbase;
        *z1 = A.zmid0;
    } else {
        *z0 = A.zmid1;
        *z1 = A.zend;
    }
}

__host__ __device__ __forceinline__ int chunk_count(const StepArgs &A)
{
    return (A.zmid0 > A.zbase ? 1 : 0) + (A.zmid1 - A.zmid0 + A.zchunk - 1) / A.zchunk + (A.zend > A.zmid1 ? 1 : 0);
}

// The body of one CTA.  kEdge = false is the interior form: the CTA's tile
// with its 4-node x / y halo and its z range with 4 planes either side lie
// inside the grid and outside every CPML slab, so it needs no memory
// variables, no coefficient tables and no masks at the grid edge.  The same
// arithmetic in the same order runs in both forms.  kStag selects the
// staggered (Yee) neighbour sets; the velocity CPML then reads the half-node
// coefficients sCxv, sCyv, A.cbv.. (the node tables otherwise).  kLocal
// takes b and a of every slab node from the per-node tables A.lb, A.la
// (local-velocity grading; 1/kappa stays the 1D table).
// Launch order of the tiles within a z-chunk row: the tiles of the columns
// that meet the x layers come first (row-major), then the others.  Those
// tiles carry the x memory variables and run slower than their neighbours;
// started first, they stay level with them along z, so that the halo lines
// both read are still in L2 (row-major order alone let them fall behind).
__device__ __forceinline__ int tile_of_block(const StepArgs &A, int b)
{
    const int e = A.xcol_lo + A.xcol_hi, m = A.tiles_x - e;
    if (e == 0)
        return b;
    if (b < e * A.tiles_y) {
        const int k = b % e;
        return (b / e) * A.tiles_x + (k < A.xcol_lo ? k : m + k);
    }
    b -= e * A.tiles_y;
    return (b / m) * A.tiles_x + A.xcol_lo + b % m;
}

template <typename T, bool kEdge, bool kRho, bool kStag, bool kLocal>
__device__ __forceinline__ void step_body(const CUtensorMap &mP, const CUtensorMap &mPq, const CUtensorMap &mVX,
                                          const CUtensorMap &mVY, const CUtensorMap &mVZ, const CUtensorMap &mK,
                                          const StepArgs &A, int z0, int z1, unsigned char *smem,
                                          float (*sCx)[TX + 8], float (*sCy)[TY + 8],
                                          float (*sCxv)[TX + 8], float (*sCyv)[TY + 8])
{
    using L = StageLayout<T>;
    constexpr bool kSplit = sizeof(T) == 2;   // see dnb
    float *svx = reinterpret_cast<float *>(smem + NSTAGE * L::BYTES);
    float *svy = svx + L::SVX_FLOATS;
    uint64_t *bar = reinterpret_cast<uint64_t *>(svy + L::SVY_FLOATS);

    const Geom &G = A.g;
    const int tid = threadIdx.x;
    const int tx = tid % (TX / 4), ty = tid / (TX / 4);
    const int tile = tile_of_block(A, blockIdx.x);
    const int x0 = (tile % A.tiles_x) * TX, y0 = (tile / A.tiles_x) * TY;
    const int shot = blockIdx.z;
    const int gx = x0 + 4 * tx, gy = y0 + ty;
    const int niter = z1 - z0 + 8;

    Coef C;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        C.cp[l] = make_float2(A.c[l], A.c[l]);
        C.cn[l] = make_float2(-A.c[l], -A.c[l]);
    }
    const float2 ndtr = make_float2(-A.dtr, -A.dtr);
    const bool aniso = A.kr[0] != 1.f || A.kr[1] != 1.f || A.kr[2] != 1.f;   // CTA-uniform

    const long long fofs = (long long)shot * G.vol;
    const T *p_in = reinterpret_cast<const T *>(A.p_in) + fofs;
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

    for (int i = tid; kEdge && i < 3 * (TX + 8); i += NTHREADS) {
        const int c = i / (TX + 8), x = x0 - 4 + i % (TX + 8);
        const bool in = x >= 0 && x < G.nx && in_slab(x, G.nx, G.lo[0], G.hi[0]);
        sCx[c][i % (TX + 8)] = in ? (c == 0 ? A.cb[0][x] : (c == 1 ? A.ca[0][x] : A.ck[0][x])) : (c == 2 ? 1.f : 0.f);
    }
    for (int i = tid; kEdge && i < 3 * (TY + 8); i += NTHREADS) {
        const int c = i / (TY + 8), y = y0 - 4 + i % (TY + 8);
        const bool in = y >= 0 && y < G.ny && in_slab(y, G.ny, G.lo[1], G.hi[1]);
        sCy[c][i % (TY + 8)] = in ? (c == 0 ? A.cb[1][y] : (c == 1 ? A.ca[1][y] : A.ck[1][y])) : (c == 2 ? 1.f : 0.f);
    }
    for (int i = tid; kStag && kEdge && i < 3 * (TX + 8); i += NTHREADS) {
        const int c = i / (TX + 8), x = x0 - 4 + i % (TX + 8);
        const bool in = x >= 0 && x < G.nx && in_slab(x, G.nx, G.lo[0], G.hi[0]);
        sCxv[c][i % (TX + 8)] = in ? (c == 0 ? A.cbv[0][x] : (c == 1 ? A.cav[0][x] : A.ckv[0][x])) : (c == 2 ? 1.f : 0.f);
    }
    for (int i = tid; kStag && kEdge && i < 3 * (TY + 8); i += NTHREADS) {
        const int c = i / (TY + 8), y = y0 - 4 + i % (TY + 8);
        const bool in = y >= 0 && y < G.ny && in_slab(y, G.ny, G.lo[1], G.hi[1]);
        sCyv[c][i % (TY + 8)] = in ? (c == 0 ? A.cbv[1][y] : (c == 1 ? A.cav[1][y] : A.ckv[1][y])) : (c == 2 ? 1.f : 0.f);
    }

    // validity of the 4 own nodes (ghost nodes beyond the grid hold 0)
    const bool row_ok = gy < G.ny && gx < G.nxp;
    float mk[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        mk[i] = ((gx + i < G.nx) && (gy < G.ny)) ? 1.f : 0.f;
    const V4 mask = V4{make_float2(mk[0], mk[1]), make_float2(mk[2], mk[3])};
    const bool full_tile = !kEdge || ((x0 + TX <= G.nx) && (y0 + TY <= G.ny));
    const long long rowofs = (long long)gy * G.nxp + gx;

    // which memory variables this thread touches (own vector, halo vector)
    const bool own_x = kEdge && G.w[0] > 0 && gy < G.ny && gx < G.nx && (gx < G.lo[0] || gx + 3 >= G.nx - G.hi[0]);
    const bool own_y = kEdge && G.w[1] > 0 && row_ok && in_slab(gy, G.ny, G.lo[1], G.hi[1]);

    // halo task of this thread: one pair of nodes.  Threads 0..127: the y
    // halo (8 rows x 16 pairs), threads 128..255: the x halo (32 rows x 2
    // pairs on each side).  Every thread then computes 1.5 vectors of v'.
    static_assert(TX == 32 && TY == 32 && NTHREADS == 256, "halo pairs assume 32x32 tiles and 256 threads");
    const bool do_yhalo = tid < 128;
    const int yh_r = (tid / 16) & 7;
    const int yh_y = yh_r < 4 ? y0 - 4 + yh_r : y0 + TY + (yh_r - 4);
    const int yh_x = x0 + 2 * (tid % 16);
    const int xh_k = tid & 3;
    const int xh_x = xh_k < 2 ? x0 - 4 + 2 * xh_k : x0 + TX + 2 * (xh_k - 2);
    const int xh_y = y0 + ((tid - 128) >> 2);
    const bool yh_in = yh_y >= 0 && yh_y < G.ny;
    const bool halo_psi_y = kEdge && do_yhalo && G.w[1] > 0 && yh_in && yh_x < G.nxp && in_slab(yh_y, G.ny, G.lo[1], G.hi[1]);
    const bool halo_psi_x = kEdge && !do_yhalo && G.w[0] > 0 && xh_y < G.ny && xh_x >= 0 && xh_x < G.nx &&
                            (xh_x < G.lo[0] || xh_x + 1 >= G.nx - G.hi[0]);
    const bool slab_thread = own_x || own_y || halo_psi_x || halo_psi_y;

    // source of this shot
    const int sz = A.src ? A.src[3 * shot] : -1, sy = A.src ? A.src[3 * shot + 1] : -1,
              sx = A.src ? A.src[3 * shot + 2] : -1;
    const float wsrc = (A.src && A.t < A.nt_w) ? A.sscale * A.wavelet[(long long)shot * A.nt_w + A.t] : 0.f;
    const bool src_here = A.src && sy == gy && sx >= gx && sx < gx + 4 && sz >= z0 && sz < z1;
    // receivers of this tile (sorted by z)
    // receivers of this tile: rec_off[tile * nz + z] .. [+ 1] are those on plane z
    const bool rec_on = A.traces != nullptr && A.nrec > 0 && A.t < A.nt_max;
    const int *roff = A.rec_off + (long long)tile * G.nz;

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

    // Issue the loads of iteration `it` into its stage (thread 0 only).  The
    // failure test leaves one stage of CTA (0, 0, 0) without its copies, so
    // that the bounded wait on it gives up (the kernel then reports
    // ERR_TIMEOUT, drains its copies in flight and returns).
    auto issue = [&](int it) {
        if (it == A.fault_it && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)
            return;
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

    // register queues: pq[j] = p(t + j), vzq[j] = v'_z(t - 4 + j)
    V4 pq[9], vzq[9];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int z = z0 - 8 + k;
        pq[k] = v4zero();
        if (z >= 0 && row_ok)
            pq[k] = to_v4(Io<T>::ldg4(p_in + (long long)z * G.plane + rowofs));
        vzq[k] = v4zero();
    }
    pq[8] = v4zero();
    vzq[8] = v4zero();

    for (int it = 0; it < niter; ++it) {
        const int t = z0 - 8 + it;
        const int zv = t + 4;
        const bool active = t >= z0;
        const unsigned char *S = smem + (it % NSTAGE) * L::BYTES;

        const bool zs_v = kEdge && row_ok && zv >= 0 && zv < G.nz && in_slab(zv, G.nz, G.lo[2], G.hi[2]);
        const bool zs_p = kEdge && active && row_ok && in_slab(t, G.nz, G.lo[2], G.hi[2]);

        // L2 prefetch of the memory variables of the next plane, so that the
        // slab loads of the next iteration do not wait on HBM
        if (kEdge) {
            const int tn = t + 1, zn = zv + 1;
            if (row_ok && zn < G.nz && zn >= 0 && in_slab(zn, G.nz, G.lo[2], G.hi[2])) {
                const long long i = slab_index(G, 2, zn, gy, gx);
                prefetch_l2(psiv_in[2] + i);
                if (kLocal) {
                    prefetch_l2(A.lb[2] + i);
                    prefetch_l2(A.la[2] + i);
                }
            }
            if (tn >= z0 && tn < z1) {
                if (row_ok && in_slab(tn, G.nz, G.lo[2], G.hi[2]))
                    prefetch_l2(psip[2] + slab_index(G, 2, tn, gy, gx));
                if (slab_thread) {
                    if (own_x) {
                        const long long i = slab_index(G, 0, tn, gy, gx);
                        prefetch_l2(psiv_in[0] + i);
                        prefetch_l2(psip[0] + i);
                        if (kLocal) {
                            prefetch_l2(A.lb[0] + i);
                            prefetch_l2(A.la[0] + i);
                        }
                    }
                    if (own_y) {
                        const long long i = slab_index(G, 1, tn, gy, gx);
                        prefetch_l2(psiv_in[1] + i);
                        prefetch_l2(psip[1] + i);
                        if (kLocal) {
                            prefetch_l2(A.lb[1] + i);
                            prefetch_l2(A.la[1] + i);
                        }
                    }
                    if (halo_psi_y)
                        prefetch_l2(psiv_in[1] + slab_index(G, 1, tn, yh_y, yh_x));
                    if (halo_psi_x)
                        prefetch_l2(psiv_in[0] + slab_index(G, 0, tn, xh_y, xh_x));
                }
            }
        }

        // -dt vscale / rho (variable density): this plane's factors are
        // loaded before the wait, so that their latency overlaps it, and the
        // next plane's go into L2
        V4 nbo = v4zero(), nbz = v4zero();
        float2 nbh = make_float2(0.f, 0.f);
        if (kRho) {
            if (t >= z0)
                nbo = ld_nbr(A.nbr, (long long)t * G.plane + rowofs, row_ok);
            if (zv >= 0 && zv < G.nz)
                nbz = ld_nbr(A.nbr, (long long)zv * G.plane + rowofs, row_ok);
            if (t >= z0) {
                const int hy = do_yhalo ? yh_y : xh_y, hx = do_yhalo ? yh_x : xh_x;
                const bool hin = do_yhalo ? (yh_in && yh_x < G.nxp) : (xh_y < G.ny && xh_x >= 0 && xh_x < G.nxp);
                const long long ho = (long long)hy * G.nxp + hx;
                if (hin) {
                    nbh = __ldg(reinterpret_cast<const float2 *>(A.nbr + (long long)t * G.plane + ho));
                    if (t + 1 < z1)
                        prefetch_l2(A.nbr + (long long)(t + 1) * G.plane + ho);
                }
            }
            if (row_ok) {
                if (t + 1 >= z0 && t + 1 < z1)
                    prefetch_l2(A.nbr + (long long)(t + 1) * G.plane + rowofs);
                if (zv + 1 >= 0 && zv + 1 < G.nz)
                    prefetch_l2(A.nbr + (long long)(zv + 1) * G.plane + rowofs);
            }
        }
        const bool ok = mbar_wait_bounded(&bar[it % NSTAGE], (it / NSTAGE) & 1, WAIT_LIMIT);

        // ---- z block: p(t + 8) into the queue (TMA zero-fills nodes beyond the
        // grid), D_z p and v'_z at plane t + 4, D_z v'_z at plane t, and p(t)
        const V4 pnew = (ok && t + 8 < G.nz) ? lds<T>(S + L::OFF_PQ, ty * TX + 4 * tx) : v4zero();
        auto zvel = [&](V4 gz) -> V4 {
            V4 vzn = v4zero();
            if (ok && zv >= 0 && zv < G.nz) {
                const bool owned = zv >= z0 && zv < z1;
                if (zs_v) {
                    const long long izv = slab_index(G, 2, zv, gy, gx);
                    const V4 psvz = ldg_v4(psiv_in[2] + izv);
                    const V4 b = kLocal ? ldc4(A.lb[2] + izv) : splat4(__ldg(A.cbv[2] + zv)),
                             a = kLocal ? ldc4(A.la[2] + izv) : splat4(__ldg(A.cav[2] + zv)),
                             k = splat4(__ldg(A.ckv[2] + zv));
                    if (owned && stape[2])
                        tape4(stape[2], izv, 0, gz, psvz);
                    const V4 pn = cpml4(gz, psvz, b, a, k);
                    if (owned)
                        st_out(psiv_out[2] + izv, to_f4(pn));
                }
                if (kRho)
                    vzn = fmav(nbz, gz, lds<T>(S + L::OFF_VZ, ty * TX + 4 * tx));
                else
                    vzn = fma4(ndtr, gz, lds<T>(S + L::OFF_VZ, ty * TX + 4 * tx));
                if (owned && row_ok)
                    st_out(v_out[2] + (long long)zv * G.plane + rowofs, to_f4(vzn));
            }
            return vzn;
        };
        V4 pt, hz4;
        zblock<kStag, kSplit>(pq, vzq, pnew, C, zvel, pt, hz4);

        if (ok && active) {
            const unsigned char *Sp = S + L::OFF_P;   // p plane, origin (x0 - 8, y0 - 8)
            const long long pofs = (long long)t * G.plane + rowofs;
            // ---- v'_x, own nodes
            {
                const int lrow = (ty + 8) * L::PW, lx = 4 * tx + 8;
                const V4 u = lds<T>(Sp, lrow + lx - 4), v = lds<T>(Sp, lrow + lx), w = lds<T>(Sp, lrow + lx + 4);
                V4 g = kStag ? sdf4(u, v, w, C) : dx4(u, v, w, C);
                if (own_x) {
                    const int cx = 4 * tx + 4;
                    const long long ix = slab_index(G, 0, t, gy, gx);
                    const V4 psvx = ldg_v4(psiv_in[0] + ix);
                    if (stape[0])
                        tape4(stape[0], ix, 0, g, psvx);
                    const V4 pn = cpml4(g, psvx, kLocal ? ldc4(A.lb[0] + ix) : ldsf(&sCxv[0][cx]),
                                        kLocal ? ldc4(A.la[0] + ix) : ldsf(&sCxv[1][cx]), ldsf(&sCxv[2][cx]));
                    st_out(psiv_out[0] + ix, to_f4(pn));
                }
                V4 vn = kRho ? fmav(nbo, g, lds<T>(S + L::OFF_VX, ty * L::VXW + 4 * tx + 8))
                             : fma4(ndtr, g, lds<T>(S + L::OFF_VX, ty * L::VXW + 4 * tx + 8));
                if (!full_tile)
                    vn = mul4(vn, mask);
                if (row_ok)
                    st_out(v_out[0] + pofs, to_f4(vn));
                stsf(svx + ty * L::SVXW + 4 * tx + 4, vn);
            }
            // ---- v'_y, own nodes
            {
                const int lx = 4 * tx + 8, ly = ty + 8;
                V4 m[4], p[4];
#pragma unroll
                for (int l = 1; l <= 4; ++l) {
                    m[l - 1] = lds<T>(Sp, (ly - l + (kStag ? 1 : 0)) * L::PW + lx);
                    p[l - 1] = lds<T>(Sp, (ly + l) * L::PW + lx);
                }
                V4 g = dnb<kSplit>(m, p, C);
                if (own_y) {
                    const long long iy = slab_index(G, 1, t, gy, gx);
                    const V4 psvy = ldg_v4(psiv_in[1] + iy);
                    if (stape[1])
                        tape4(stape[1], iy, 0, g, psvy);
                    const V4 pn = cpml4(g, psvy, kLocal ? ldc4(A.lb[1] + iy) : splat4(sCyv[0][ty + 4]),
                                        kLocal ? ldc4(A.la[1] + iy) : splat4(sCyv[1][ty + 4]), splat4(sCyv[2][ty + 4]));
                    st_out(psiv_out[1] + iy, to_f4(pn));
                }
                V4 vn = kRho ? fmav(nbo, g, lds<T>(S + L::OFF_VY, (ty + 4) * TX + 4 * tx))
                             : fma4(ndtr, g, lds<T>(S + L::OFF_VY, (ty + 4) * TX + 4 * tx));
                if (!full_tile)
                    vn = mul4(vn, mask);
                if (row_ok)
                    st_out(v_out[1] + pofs, to_f4(vn));
                stsf(svy + (ty + 4) * TX + 4 * tx, vn);
            }
            // ---- halos (recomputed, not stored): one pair of nodes per thread
            if (do_yhalo) {
                const int ly = yh_y - y0 + 8, lx = yh_x - x0 + 8;
                float2 m[4], p[4];
#pragma unroll
                for (int l = 1; l <= 4; ++l) {
                    m[l - 1] = lds2<T>(Sp, (ly - l + (kStag ? 1 : 0)) * L::PW + lx);
                    p[l - 1] = lds2<T>(Sp, (ly + l) * L::PW + lx);
                }
                float2 g = dnb2<kSplit>(m, p, C);
                const int r = yh_y - y0 + 4;
                if (halo_psi_y) {
                    const long long ih = slab_index(G, 1, t, yh_y, yh_x);
                    const float2 psh = Io<T>::ld2(psiv_in[1] + ih);
                    cpml2(g, psh, kLocal ? ldc2(A.lb[1] + ih) : make_float2(sCyv[0][r], sCyv[0][r]),
                          kLocal ? ldc2(A.la[1] + ih) : make_float2(sCyv[1][r], sCyv[1][r]),
                          make_float2(sCyv[2][r], sCyv[2][r]));
                }
                float2 vn = fma2(kRho ? nbh : ndtr, g, lds2<T>(S + L::OFF_VY, r * TX + (yh_x - x0)));
                if (kEdge) {
                    vn.x = (yh_in && yh_x < G.nx) ? vn.x : 0.f;
                    vn.y = (yh_in && yh_x + 1 < G.nx) ? vn.y : 0.f;
                }
                *reinterpret_cast<float2 *>(svy + r * TX + (yh_x - x0)) = vn;
            } else {
                const int lrow = (xh_y - y0 + 8) * L::PW, lx = xh_x - x0 + 8;
                const float2 P0 = lds2<T>(Sp, lrow + lx - 4), P1 = lds2<T>(Sp, lrow + lx - 2), P2 = lds2<T>(Sp, lrow + lx),
                             P3 = lds2<T>(Sp, lrow + lx + 2), P4 = lds2<T>(Sp, lrow + lx + 4);
                float2 g = kStag ? sdf2(P0, P1, P2, P3, P4, C) : dx2(P0, P1, P2, P3, P4, C);
                const int cx = xh_x - x0 + 4;
                if (halo_psi_x) {
                    const long long ih = slab_index(G, 0, t, xh_y, xh_x);
                    const float2 psh = Io<T>::ld2(psiv_in[0] + ih);
                    cpml2(g, psh, kLocal ? ldc2(A.lb[0] + ih) : *reinterpret_cast<const float2 *>(&sCxv[0][cx]),
                          kLocal ? ldc2(A.la[0] + ih) : *reinterpret_cast<const float2 *>(&sCxv[1][cx]),
                          *reinterpret_cast<const float2 *>(&sCxv[2][cx]));
                }
                float2 vn = fma2(kRho ? nbh : ndtr, g, lds2<T>(S + L::OFF_VX, (xh_y - y0) * L::VXW + lx));
                if (kEdge) {
                    vn.x = (xh_y < G.ny && xh_x >= 0 && xh_x < G.nx) ? vn.x : 0.f;
                    vn.y = (xh_y < G.ny && xh_x + 1 >= 0 && xh_x + 1 < G.nx) ? vn.y : 0.f;
                }
                *reinterpret_cast<float2 *>(svx + (xh_y - y0) * L::SVXW + cx) = vn;
            }
        }

        // all v' of plane t are in shared memory; stop together on a timeout
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
            const float *sxr = svx + ty * L::SVXW + 4 * tx;
            V4 hx4 = kStag ? sdb4(ldsf(sxr), ldsf(sxr + 4), ldsf(sxr + 8), C)
                           : dx4(ldsf(sxr), ldsf(sxr + 4), ldsf(sxr + 8), C);
            V4 hy4;
            {
                V4 m[4], p[4];
#pragma unroll
                for (int l = 1; l <= 4; ++l) {
                    m[l - 1] = ldsf(svy + (ty + 4 - l) * TX + 4 * tx);
                    p[l - 1] = ldsf(svy + (ty + 4 + l - (kStag ? 1 : 0)) * TX + 4 * tx);
                }
                hy4 = dnb<kSplit>(m, p, C);
            }
            if (own_x) {
                const int cx = 4 * tx + 4;
                const long long ix = slab_index(G, 0, t, gy, gx);
                const V4 pspx = ldg_v4(psip[0] + ix);
                if (stape[0])
                    tape4(stape[0], ix, 2, hx4, pspx);
                const V4 pn = cpml4(hx4, pspx, kLocal ? ldc4(A.lb[0] + ix) : ldsf(&sCx[0][cx]),
                                    kLocal ? ldc4(A.la[0] + ix) : ldsf(&sCx[1][cx]), ldsf(&sCx[2][cx]));
                st_out(psip[0] + ix, to_f4(pn));
            }
            if (own_y) {
                const long long iy = slab_index(G, 1, t, gy, gx);
                const V4 pspy = ldg_v4(psip[1] + iy);
                if (stape[1])
                    tape4(stape[1], iy, 2, hy4, pspy);
                const V4 pn = cpml4(hy4, pspy, kLocal ? ldc4(A.lb[1] + iy) : splat4(sCy[0][ty + 4]),
                                    kLocal ? ldc4(A.la[1] + iy) : splat4(sCy[1][ty + 4]), splat4(sCy[2][ty + 4]));
                st_out(psip[1] + iy, to_f4(pn));
            }
            if (zs_p) {
                const long long izp = slab_index(G, 2, t, gy, gx);
                const V4 pspz = ldg_v4(psip[2] + izp);
                if (stape[2])
                    tape4(stape[2], izp, 2, hz4, pspz);
                const V4 pn = cpml4(hz4, pspz, kLocal ? ldc4(A.lb[2] + izp) : splat4(__ldg(A.cb[2] + t)),
                                    kLocal ? ldc4(A.la[2] + izp) : splat4(__ldg(A.ca[2] + t)), splat4(__ldg(A.ck[2] + t)));
                st_out(psip[2] + izp, to_f4(pn));
            }
            // nkdt holds -dt K / vscale (zero beyond the grid)
            const V4 nkd = ldsf(reinterpret_cast<const float *>(S + L::OFF_K) + ty * TX + 4 * tx);
            // elliptic anisotropy weights the axes (A.kr = 1, 1, 1 when isotropic)
            const V4 sb = aniso ? add4(add4(mul4(splat4(A.kr[0]), hx4), mul4(splat4(A.kr[1]), hy4)),
                                       mul4(splat4(A.kr[2]), hz4))
                                : add4(add4(hx4, hy4), hz4);
            V4 pn = V4{fma2(nkd.a, sb.a, pt.a), fma2(nkd.b, sb.b, pt.b)};
            if (src_here && t == sz) {
                const int i = sx - gx;   // select, not a dynamic register index
                pn.a.x += (i == 0) ? wsrc : 0.f;
                pn.a.y += (i == 1) ? wsrc : 0.f;
                pn.b.x += (i == 2) ? wsrc : 0.f;
                pn.b.y += (i == 3) ? wsrc : 0.f;
            }
            if (row_ok) {
                const long long o = (long long)t * G.plane + rowofs;
                st_out(reinterpret_cast<T *>(A.p_out) + fofs + o, to_f4(pn));
                if (A.s_tape)
                    stsf(A.s_tape + fofs + o, sb);
            }
            if (rec_on) {
                const int r0 = __ldg(roff + t), r1 = __ldg(roff + t + 1);
                if (r0 < r1) {
                    // the plane's new p goes to this stage's K slots, which each
                    // thread has just read for its own nodes; then the CTA reads
                    // the plane's receivers together
                    float *pl = reinterpret_cast<float *>(smem + (it % NSTAGE) * L::BYTES + L::OFF_K);
                    stsf(pl + ty * TX + 4 * tx, pn);
                    __syncthreads();
                    for (int r = r0 + tid; r < r1; r += NTHREADS) {
                        const int4 q = A.rec[r];
                        // read back through the storage type so traces equal the stored state
                        T tmp = T(pl[(q.y - y0) * TX + (q.z - x0)]);
                        A.traces[((long long)shot * A.nt_max + A.t) * A.nrec + q.w] = A.inv_sscale * Io<T>::ld1(&tmp);
                    }
                }
            }
        }
        __syncthreads();
        if (tid == 0 && it + NSTAGE < niter) {
            fence_proxy_async_smem();
            issue(it + NSTAGE);
        }
    }
}

template <typename T, bool kRho, bool kStag, bool kLocal>
__global__ void __launch_bounds__(NTHREADS, kMinBlocks)
    fdtd_step_kernel(const __grid_constant__ CUtensorMap mP, const __grid_constant__ CUtensorMap mPq,
                     const __grid_constant__ CUtensorMap mVX, const __grid_constant__ CUtensorMap mVY,
                     const __grid_constant__ CUtensorMap mVZ, const __grid_constant__ CUtensorMap mK,
                     const StepArgs A)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    // CPML coefficients (b, a, 1/kappa) of the tile's x range [x0-4, x0+TX+4)
    // and y range [y0-4, y0+TY+4); 0, 0, 1 outside the slabs and the grid
    __shared__ __align__(16) float sCx[3][TX + 8];
    __shared__ __align__(16) float sCy[3][TY + 8];
    // the staggered form's velocity coefficients (half-node depths)
    __shared__ __align__(16) float sCxv[kStag ? 3 : 1][TX + 8];
    __shared__ __align__(16) float sCyv[kStag ? 3 : 1][TY + 8];
    float (*vx)[TX + 8] = kStag ? sCxv : sCx;
    float (*vy)[TY + 8] = kStag ? sCyv : sCy;
    const Geom &G = A.g;
    const int tile = tile_of_block(A, blockIdx.x);
    const int x0 = (tile % A.tiles_x) * TX, y0 = (tile / A.tiles_x) * TY;
    int z0, z1;
    chunk_range(A, blockIdx.y, &z0, &z1);
    const bool interior = x0 - 4 >= G.lo[0] && x0 + TX + 4 <= G.nx - G.hi[0] && y0 - 4 >= G.lo[1] &&
                          y0 + TY + 4 <= G.ny - G.hi[1] && z0 - 4 >= G.lo[2] && z1 + 4 <= G.nz - G.hi[2];
    if (interior)
        step_body<T, false, kRho, kStag, false>(mP, mPq, mVX, mVY, mVZ, mK, A, z0, z1, smem, sCx, sCy, vx, vy);
    else
        step_body<T, true, kRho, kStag, kLocal>(mP, mPq, mVX, mVY, mVZ, mK, A, z0, z1, smem, sCx, sCy, vx, vy);
}

template <typename T, bool kRho, bool kStag, bool kLocal>
static cudaError_t launch_step_tr(const fdtd_ctx *c, const StepArgs &a, int set, cudaStream_t stream)
{
    using L = StageLayout<T>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(fdtd_step_kernel<T, kRho, kStag, kLocal>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
        if (e != cudaSuccess)
            return e;
        attr_done = true;
    }
    dim3 grid(c->tiles_x * c->tiles_y, chunk_count(a), c->d.nshots);
    fdtd_step_kernel<T, kRho, kStag, kLocal><<<grid, NTHREADS, L::SMEM, stream>>>(
        c->maps[set][0], c->maps[set][1], c->maps[set][2], c->maps[set][3], c->maps[set][4], c->mapK, a);
    return cudaGetLastError();
}

// a.nbr selects the variable-density form, c->staggered the staggered one
// (FP32 storage and constant density only), a.lb[0] the local grading (FP32
// storage, collocated); the API enforces these combinations
template <typename T>
static cudaError_t launch_step_t(const fdtd_ctx *c, const StepArgs &a, int set, cudaStream_t stream)
{
    if constexpr (std::is_same<T, float>::value) {
        if (c->staggered)
            return (a.nbr || a.lb[0]) ? cudaErrorInvalidValue : launch_step_tr<T, false, true, false>(c, a, set, stream);
        if (a.lb[0])
            return a.nbr ? launch_step_tr<T, true, false, true>(c, a, set, stream)
                         : launch_step_tr<T, false, false, true>(c, a, set, stream);
    }
    return a.nbr ? launch_step_tr<T, true, false, false>(c, a, set, stream)
                 : launch_step_tr<T, false, false, false>(c, a, set, stream);
}

// One step over z in [a.zbase, a.zend) on `stream`; `set` is the ping-pong
// set holding the input state.
cudaError_t launch_step(const fdtd_ctx *c, const StepArgs &a, int set, cudaStream_t stream)
{
    switch (c->d.storage) {
    case FDTD_F16:
        return launch_step_t<__half>(c, a, set, stream);
    case FDTD_BF16:
        return launch_step_t<__nv_bfloat16>(c, a, set, stream);
    default:
        return launch_step_t<float>(c, a, set, stream);
    }
}

template <typename T>
static int occupancy_t(int *blocks)
{
    using L = StageLayout<T>;
    cudaFuncSetAttribute(fdtd_step_kernel<T, false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fdtd_step_kernel<T, false, false, false>, NTHREADS, L::SMEM) ==
                   cudaSuccess
               ? 0
               : -1;
}

int step_occupancy(int storage, int *blocks)
{
    switch (storage) {
    case FDTD_F16:
        return occupancy_t<__half>(blocks);
    case FDTD_BF16:
        return occupancy_t<__nv_bfloat16>(blocks);
    default:
        return occupancy_t<float>(blocks);
    }
}

}  // namespace fdtd

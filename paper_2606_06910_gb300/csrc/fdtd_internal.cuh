// Internal declarations of libfdtd: context, kernel argument blocks, storage
// traits and the inline-PTX helpers (mbarrier, TMA) used by the kernels.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fdtd.h"

namespace fdtd {

// Forward tile: TX x TY nodes in (x, y) per CTA, each thread owns 4
// consecutive x nodes of one row; the CTA marches a z range.
constexpr int TX = 32;
constexpr int TY = 32;
constexpr int NTHREADS = (TX / 4) * TY;   // 256
constexpr int NSTAGE = 3;                 // TMA pipeline depth (planes in flight)

// Weights a_1..a_4 of the centred radius-4 first derivative (paper Sec. 3.1
// leaves them unprinted): the unique antisymmetric weights that differentiate
// polynomials up to degree 8 exactly.
constexpr double kWeights[4] = {4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0};

// Weights c_1..c_4 of the staggered radius-4 first derivative (the Yee form of
// Sec. 3.1: offsets 1/2, 3/2, 5/2, 7/2), exact for polynomials up to degree 7.
constexpr double kStagWeights[4] = {1225.0 / 1024.0, -245.0 / 3072.0, 49.0 / 5120.0, -5.0 / 7168.0};

// device error word bits
constexpr unsigned ERR_TIMEOUT = 1u;
constexpr unsigned ERR_NONFINITE = 2u;

// bounded spin on an mbarrier: 2^18 polls (about a second on GB300, where a
// poll that finds the phase incomplete takes about 4 us) before giving up; a
// plane's copies normally land within microseconds
constexpr unsigned WAIT_LIMIT = 1u << 18;
constexpr unsigned WAIT_LIMIT_DRAIN = 1u << 15;

struct F4 {
    float v[4];
};

// ---------------------------------------------------------------------------
// storage traits: load/store 4 consecutive elements, convert to/from FP32
// ---------------------------------------------------------------------------
template <typename T>
struct Io;

template <>
struct Io<float> {
    static __device__ __forceinline__ F4 ld4(const float *p)
    {
        float4 q = *reinterpret_cast<const float4 *>(p);
        return F4{{q.x, q.y, q.z, q.w}};
    }
    static __device__ __forceinline__ F4 ldg4(const float *p)
    {
        float4 q = __ldg(reinterpret_cast<const float4 *>(p));
        return F4{{q.x, q.y, q.z, q.w}};
    }
    static __device__ __forceinline__ void st4(float *p, const F4 &v)
    {
        *reinterpret_cast<float4 *>(p) = make_float4(v.v[0], v.v[1], v.v[2], v.v[3]);
    }
    // store that is not read again soon (L2 evict-first)
    static __device__ __forceinline__ void st4s(float *p, const F4 &v)
    {
        __stcs(reinterpret_cast<float4 *>(p), make_float4(v.v[0], v.v[1], v.v[2], v.v[3]));
    }
    static __device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    static __device__ __forceinline__ float ld1(const float *p) { return *p; }
    static __device__ __forceinline__ void st1(float *p, float v) { *p = v; }
};

template <>
struct Io<__half> {
    static __device__ __forceinline__ F4 from_u2(uint2 u)
    {
        __half2 a = *reinterpret_cast<__half2 *>(&u.x);
        __half2 b = *reinterpret_cast<__half2 *>(&u.y);
        float2 fa = __half22float2(a), fb = __half22float2(b);
        return F4{{fa.x, fa.y, fb.x, fb.y}};
    }
    static __device__ __forceinline__ F4 ld4(const __half *p)
    {
        return from_u2(*reinterpret_cast<const uint2 *>(p));
    }
    static __device__ __forceinline__ F4 ldg4(const __half *p)
    {
        return from_u2(__ldg(reinterpret_cast<const uint2 *>(p)));
    }
    static __device__ __forceinline__ uint2 to_u2(const F4 &v)
    {
        __half2 a = __floats2half2_rn(v.v[0], v.v[1]);
        __half2 b = __floats2half2_rn(v.v[2], v.v[3]);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t *>(&a);
        u.y = *reinterpret_cast<uint32_t *>(&b);
        return u;
    }
    static __device__ __forceinline__ void st4(__half *p, const F4 &v) { *reinterpret_cast<uint2 *>(p) = to_u2(v); }
    static __device__ __forceinline__ void st4s(__half *p, const F4 &v) { __stcs(reinterpret_cast<uint2 *>(p), to_u2(v)); }
    static __device__ __forceinline__ float2 ld2(const __half *p)
    {
        return __half22float2(*reinterpret_cast<const __half2 *>(p));
    }
    static __device__ __forceinline__ float ld1(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st1(__half *p, float v) { *p = __float2half_rn(v); }
};

template <>
struct Io<__nv_bfloat16> {
    static __device__ __forceinline__ F4 from_u2(uint2 u)
    {
        __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162 *>(&u.x);
        __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162 *>(&u.y);
        float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        return F4{{fa.x, fa.y, fb.x, fb.y}};
    }
    static __device__ __forceinline__ F4 ld4(const __nv_bfloat16 *p)
    {
        return from_u2(*reinterpret_cast<const uint2 *>(p));
    }
    static __device__ __forceinline__ F4 ldg4(const __nv_bfloat16 *p)
    {
        return from_u2(__ldg(reinterpret_cast<const uint2 *>(p)));
    }
    static __device__ __forceinline__ uint2 to_u2(const F4 &v)
    {
        __nv_bfloat162 a = __floats2bfloat162_rn(v.v[0], v.v[1]);
        __nv_bfloat162 b = __floats2bfloat162_rn(v.v[2], v.v[3]);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t *>(&a);
        u.y = *reinterpret_cast<uint32_t *>(&b);
        return u;
    }
    static __device__ __forceinline__ void st4(__nv_bfloat16 *p, const F4 &v)
    {
        *reinterpret_cast<uint2 *>(p) = to_u2(v);
    }
    static __device__ __forceinline__ void st4s(__nv_bfloat16 *p, const F4 &v)
    {
        __stcs(reinterpret_cast<uint2 *>(p), to_u2(v));
    }
    static __device__ __forceinline__ float2 ld2(const __nv_bfloat16 *p)
    {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
    }
    static __device__ __forceinline__ float ld1(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st1(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

// ---------------------------------------------------------------------------
// inline PTX: shared-memory mbarrier and TMA (cp.async.bulk.tensor)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar`, giving up after `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, unsigned limit)
{
    for (unsigned i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity))
            return true;
    return false;
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2, int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// bring the line holding p into L2; no register result, no wait
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---------------------------------------------------------------------------
// geometry shared by kernels and host
// ---------------------------------------------------------------------------
// Memory variables live only in their slabs.  y and z slabs are whole rows /
// planes: [nz][lo+hi][nxp] and [lo+hi][ny][nxp].  The x slabs are short row
// segments: [nz][ny][w0] with the low face at compact x = x and the high face
// at compact x = xhi + (x - (nx - hi)), where xhi keeps compact x congruent to
// x modulo 4 (16-byte vectors of 4 nodes stay aligned) and leaves at least 4
// unused entries between the faces and after the high face, so a vector that
// straddles a slab edge reads or writes only padding outside the slab.
struct Geom {
    int nx, ny, nz, nxp;     // nodes, padded row pitch (elements, multiple of 8)
    long long plane;         // ny * nxp
    long long vol;           // nz * plane (elements per shot)
    int lo[3], hi[3];        // CPML cells per axis (x, y, z)
    int w[3];                // compact width: w0 padded (see above), w1 = lo+hi, w2 = lo+hi
    int xhi;                 // compact x of the first high-face node
    long long slab[3];       // memory-variable elements per shot and axis
};

__host__ __device__ __forceinline__ bool in_slab(int i, int n, int lo, int hi)
{
    return i < lo || i >= n - hi;
}

// compact coordinate along the slab axis (y or z: rows / planes of the slab)
__host__ __device__ __forceinline__ int slab_coord(int i, int n, int lo, int hi)
{
    return i < lo ? i : lo + (i - (n - hi));
}

// compact x of node x in [0, nx + 3): the 4-vector starting at x & ~3 maps
// with the low face if it starts inside the low face, else with the high face
// (the x interior is at least 4 nodes wide, so no vector touches both faces)
__host__ __device__ __forceinline__ int slab_x(const Geom &g, int x)
{
    return (x & ~3) < g.lo[0] ? x : g.xhi + (x - (g.nx - g.hi[0]));
}

__host__ __device__ __forceinline__ long long slab_index(const Geom &g, int d, int z, int y, int x)
{
    if (d == 0)
        return ((long long)z * g.ny + y) * g.w[0] + slab_x(g, x);
    if (d == 1)
        return ((long long)z * g.w[1] + slab_coord(y, g.ny, g.lo[1], g.hi[1])) * g.nxp + x;
    return ((long long)slab_coord(z, g.nz, g.lo[2], g.hi[2]) * g.ny + y) * g.nxp + x;
}

// Tile columns (of width tx nodes) whose nodes or 4-node derivative reach
// meet the x layers: the first *nlo and the last *nhi columns; both 0 when the
// grid has no x layers or every column meets them.
__host__ __device__ __forceinline__ void x_layer_columns(int nx, int lo, int hi, int tx, int *nlo, int *nhi)
{
    const int ncol = (nx + tx - 1) / tx;
    int a = lo > 0 ? (lo + 4 + tx - 1) / tx : 0;
    int b = 0;
    if (hi > 0) {
        // columns c with (c + 1) tx + 4 > nx - hi, i.e. c >= floor((nx - hi - 4) / tx)
        const int first = nx - hi - 4 > 0 ? (nx - hi - 4) / tx : 0;
        b = first < ncol ? ncol - first : 0;
    }
    if (a + b >= ncol)
        a = b = 0;
    *nlo = a;
    *nhi = b;
}

// x-slab layout for a grid with nx nodes and lo / hi cells (host and tests)
__host__ __device__ __forceinline__ void x_slab_layout(int nx, int lo, int hi, int *xhi, int *w0)
{
    if (lo + hi == 0) {
        *xhi = 0;
        *w0 = 0;
        return;
    }
    const int base = (lo + 3) / 4 * 4 + 4;                 // low face + >= 4 padding
    const int r = ((nx - hi) % 4 + 4) % 4;                 // xhi == nx - hi (mod 4)
    *xhi = base + ((r - base % 4) + 4) % 4;
    *w0 = (*xhi + hi + 3) / 4 * 4 + 4;                     // high face + >= 4 padding
}

// Arguments of the fused forward step kernel (one launch = one time step).
struct StepArgs {
    Geom g;
    int tiles_x, tiles_y, zchunk;
    int xcol_lo, xcol_hi;           // tile columns at the low / high x face that meet the x layers
    int zbase, zend;                // z range of this launch: [zbase, zend)
    int zmid0, zmid1;               // chunks: [zbase, zmid0) if not empty, then zchunk planes per CTA
                                    // over [zmid0, zmid1), then [zmid1, zend) if not empty
    int t;                          // time index of this step
    const void *p_in;
    void *p_out;
    const void *v_in[3];
    void *v_out[3];
    const void *psiv_in[3];
    void *psiv_out[3];
    void *psip[3];                  // updated in place
    const float *cb[3], *ca[3], *ck[3];   // b, a, 1/kappa per node of each axis
    const float *cbv[3], *cav[3], *ckv[3];   // the same for the velocity update (half nodes when staggered)
    const float *lb[3], *la[3];     // local grading: b, a per slab node (slab layout, shared by shots), or null
    int fault_it;                   // failure test: CTA (0, 0, 0) issues no copies for this iteration (-1: none)
    float c[4];                     // a_l / h
    float dtr;                      // dt * vscale / rho (velocity update, constant density)
    const float *nbr;               // [vol] -dt * vscale / rho per node (variable density), or null
    float sscale, inv_sscale;       // stored state = sscale * physical state
    float kr[3];                    // elliptic anisotropy: axis moduli kr_d K (x, y, z)
    const int *src;                 // [nshots][3] (z, y, x)
    const float *wavelet;           // [nshots][nt_w]
    int nt_w;
    const int *rec_off;             // [tiles * nz + 1]: receivers of (tile, plane z) are rec[off .. next off)
    const int4 *rec;                // (z, y, x, r) sorted by tile, z, y, x
    int nrec, nt_max;
    float *traces;                  // [nshots][nt_max][nrec] or null
    float *s_tape;                  // [nshots][vol] pressure bracket of this step, or null
    float *slab_tape[3];            // [nshots][slab d][4] = (g, psiv_old, h, psip_old), or null
    unsigned *err;
};

}  // namespace fdtd

// The opaque context behind fdtd_ctx*.
struct fdtd_ctx {
    fdtd_desc d;
    cudaStream_t stream;
    fdtd::Geom g;
    int es;                 // bytes per stored element
    int tiles_x, tiles_y, zchunk, nzchunks;   // uniform z-chunks (adjoint kernels)
    int zmid0, zmid1, zchunk_mid;             // forward step chunks (see StepArgs::zmid0)
    int azchunk_target;                       // planes per middle chunk of the fused adjoint
    float vscale;           // stored velocity = vscale * v (impedance scaling for 16-bit)
    float vscale_req;       // fdtd_set_velocity_scale: the scale 16-bit storage uses (0: the model's maximum)
    float sscale;           // every stored field is multiplied by sscale (2^10 for FP16, else 1)
    float c_max, c_min;
    int device;             // the CUDA device current at fdtd_create
    int t;                  // time index
    int div_every;          // fdtd_set_divergence_check: every this many steps (0: off)
    double div_limit;       // energy limit in stored units (infinity: non-finite only)
    int cur;                // ping-pong buffer holding the current state
    bool model_set, cpml_set, cpml_ska;
    int nrec;
    int src_host[3 * 1024];
    // device memory carved from the caller's workspace
    unsigned char *ws;
    size_t ws_bytes;
    void *p[2], *v[3][2], *psiv[3][2], *psip[3];
    float *kdt;             // -dt K / vscale per node [nz][ny][nxp] (0 in the row padding)
    float *nbr;             // -dt vscale / rho per node (variable density), same layout
    bool var_rho;           // fdtd_set_model was given a density
    double kr[3];           // elliptic anisotropy factors (1, 1, 1: isotropic)
    bool staggered;         // the staggered (Yee) form: v_d at half nodes
    float *lcoef[3][2];     // local grading: b, a per slab node of axis d (slab layout), if reserved
    bool cpml_local_set;    // fdtd_set_cpml_local is in force
    float *coef;            // [2][3][3][nmax]: b, a, 1/kappa per axis and node, then at the half nodes
    float *wavelet;         // [nshots][nt_max]
    int nt_w;
    int *src;               // [nshots][3]
    int4 *rec;
    int *rec_off;
    float *traces;
    unsigned *err;
    double *red;            // reduction partials
    unsigned *minmax;       // vel min / max bits, invalid count
    // adjoint
    int ncp;                // checkpoint slots
    unsigned char *ckpt;    // [ncp][state]
    size_t ckpt_slot_bytes;
    float *tape_s;          // [C][nshots][vol]
    float *tape_slab[3];    // [C][nshots][slab d][4]
    float *ap, *av[3];      // adjoint mu = kdt lam_p and lam_v (FP32): the current set of apb / avb
    float *apb[2], *avb[3][2];
    int aset;
    float *apsiv[3][2], *apsip[3][2];
    int acur;
    float *gradK;           // [nshots][vol]
    float *gprof;           // [3][3][nmax]
    CUtensorMap maps[2][5]; // per ping-pong set: P halo, P queue, VX, VY, VZ
    CUtensorMap mapK;
    // adjoint (FP32, built when checkpoint slots exist), per set of mu /
    // lam_v: mu 48x48 and 32x32, lam_v_x 40x32, lam_v_y 32x40, lam_v_z 32x32
    CUtensorMap amaps[2][5];
    // temporal blocking (tblock_k > 1): one stream per step of a block, one
    // event per (step, z band); band b covers [b * tb_band, (b + 1) * tb_band)
    // and the last band runs to nz
    int tb_nb, tb_band;
    cudaStream_t tb_stream[4];
    cudaEvent_t *tb_ev;     // [tblock_k][tb_nb]
    cudaEvent_t tb_entry;
    // kernel timing (fdtd_set_timing): a pool of CUDA event pairs per kernel
    // class, recorded around each launch on its stream and folded into the
    // totals when the pool fills or the totals are read
    bool timing;
    cudaEvent_t *tev[2];    // [2 * kTimingPairs] per class, created on first use
    int tev_used[2];        // pairs recorded and not yet folded
    double t_ms[2];
    long long t_launch[2];
    char last_error[256];
};

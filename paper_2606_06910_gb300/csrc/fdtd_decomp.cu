// Halo exchange between contexts that hold parts of one grid (the domain
// decomposition of paper Sec. 3.3): fdtd_exchange copies the whole stepped
// state -- p, v, and the CPML memory variables where both sides keep them --
// over a box of the destination's grid from the matching box of the source's.
//
// The paper packs each halo into a contiguous buffer, copies it peer to peer
// and unpacks it.  Here one kernel on the destination's stream reads the
// source context's arrays directly and writes the destination's: on one GPU
// both live in the same memory; on several GPUs the same kernel would read
// the source over peer access (not built: one GPU per run).
//
// A memory variable psi_d exists only in the d-slabs of each context.  Both
// contexts are parts of one grid whose CPML sits on the global faces only, so
// a node lies in a d-slab of both or of neither, except next to an internal
// interface, where neither has one; the kernel copies psi_d where both do.
#include <algorithm>

#include "fdtd_internal.cuh"

namespace fdtd {

namespace {

struct XSide {
    Geom g;
    const unsigned char *p, *v[3], *psiv[3], *psip[3];
};

struct XDst {
    Geom g;
    unsigned char *p, *v[3], *psiv[3], *psip[3];
};

template <typename E>
__device__ __forceinline__ void cp1(unsigned char *dst, long long di, const unsigned char *src, long long si)
{
    reinterpret_cast<E *>(dst)[di] = reinterpret_cast<const E *>(src)[si];
}

// One thread per node of a box row: x from blockIdx.x / threadIdx.x, the row
// y from blockIdx.y, and (shot, z) from blockIdx.z, striding over the rest;
// E is the stored element (4 or 2 bytes).
template <typename E>
__global__ void exchange_kernel(XDst D, XSide S, int z0, int y0, int x0, int bz, int by, int bx, int sz, int sy,
                                int sx, int nshots)
{
    const int x = x0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= x0 + bx)
        return;
    const int y = y0 + blockIdx.y;
    const int xs = x + sx, ys = y + sy;
    for (int q = blockIdx.z; q < bz * nshots; q += gridDim.z) {
        const int shot = q / bz;
        const int z = z0 + (q - shot * bz);
        const int zs = z + sz;
        const long long di = shot * D.g.vol + (long long)z * D.g.plane + (long long)y * D.g.nxp + x;
        const long long si = shot * S.g.vol + (long long)zs * S.g.plane + (long long)ys * S.g.nxp + xs;
        cp1<E>(D.p, di, S.p, si);
#pragma unroll
        for (int d = 0; d < 3; ++d)
            cp1<E>(D.v[d], di, S.v[d], si);
        const int cd[3] = {x, y, z}, cs[3] = {xs, ys, zs};
        const int nd[3] = {D.g.nx, D.g.ny, D.g.nz}, ns[3] = {S.g.nx, S.g.ny, S.g.nz};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (!in_slab(cd[d], nd[d], D.g.lo[d], D.g.hi[d]) || !in_slab(cs[d], ns[d], S.g.lo[d], S.g.hi[d]))
                continue;
            const long long dj = shot * D.g.slab[d] + slab_index(D.g, d, z, y, x);
            const long long sj = shot * S.g.slab[d] + slab_index(S.g, d, zs, ys, xs);
            cp1<E>(D.psiv[d], dj, S.psiv[d], sj);
            cp1<E>(D.psip[d], dj, S.psip[d], sj);
        }
    }
}

}  // namespace

cudaError_t launch_exchange(fdtd_ctx *dst, const fdtd_ctx *src, const int box[6], const int shift[3])
{
    XDst D;
    XSide S;
    D.g = dst->g;
    S.g = src->g;
    const int cd = dst->cur, cs = src->cur;
    D.p = (unsigned char *)dst->p[cd];
    S.p = (const unsigned char *)src->p[cs];
    for (int d = 0; d < 3; ++d) {
        D.v[d] = (unsigned char *)dst->v[d][cd];
        S.v[d] = (const unsigned char *)src->v[d][cs];
        D.psiv[d] = (unsigned char *)dst->psiv[d][cd];
        S.psiv[d] = (const unsigned char *)src->psiv[d][cs];
        D.psip[d] = (unsigned char *)dst->psip[d];
        S.psip[d] = (const unsigned char *)src->psip[d];
    }
    const int bz = box[1] - box[0], by = box[3] - box[2], bx = box[5] - box[4];
    const int threads = 128;
    // rows of the box: x across threads, y across blockIdx.y (<= 65535 rows,
    // the grid's y extent), (shot, z) across blockIdx.z with a stride
    const dim3 grid((bx + threads - 1) / threads, by, (unsigned)std::min(bz * dst->d.nshots, 65535));
    if (by > 65535)
        return cudaErrorInvalidConfiguration;
    if (dst->es == 4)
        exchange_kernel<uint32_t><<<grid, threads, 0, dst->stream>>>(D, S, box[0], box[2], box[4], bz, by, bx,
                                                                      shift[0], shift[1], shift[2], dst->d.nshots);
    else
        exchange_kernel<uint16_t><<<grid, threads, 0, dst->stream>>>(D, S, box[0], box[2], box[4], bz, by, bx,
                                                                      shift[0], shift[1], shift[2], dst->d.nshots);
    return cudaGetLastError();
}

}  // namespace fdtd

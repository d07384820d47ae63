// Discrete adjoint of the fused step: the exact transpose of
//   g_d = D_d p ; psiv_d' = b psiv_d + a g_d ; v_d' = v_d - dtr (kinv g_d + psiv_d')
//   h_d = D_d v_d' ; psip_d' = b psip_d + a h_d ; p' = p - kdt sum_d kr_d (kinv h_d + psip_d')
// (CPML terms only inside the d-slab; paper Sec. 3.1-3.2), taken assignment
// by assignment in reverse.  With zero values beyond the grid the transpose
// of the centred derivative is its negative, so the adjoint is again a pair
// of radius-4 stencils, applied to pointwise-transformed adjoint fields:
//   stage A (pressure):  q = -kr_d kdt lam_p ; lam_h_d = kinv q + a (lam_psip_d + q)
//                        lam_v_d -= D_d lam_h_d ; lam_psip_d <- b (lam_psip_d + q)
//   stage B (velocity):  r = -dtr lam_v_d ; lam_g_d = kinv r + a (lam_psiv_d + r)
//                        lam_p -= sum_d D_d lam_g_d ; lam_psiv_d <- b (lam_psiv_d + r)
// and dJ/dK += -(dt / vscale) S lam_p with S the taped pressure bracket.
// (Here kdt holds the coefficient with its sign, -dt K / vscale, so q = kdt
// lam_p.)  The library stores the adjoint pressure as mu = kdt lam_p, the
// quantity stage A differentiates: q = mu, stage B updates mu -= kdt sum D
// lam_g, and dJ/dK uses lam_p = mu / kdt.
#include "fdtd_internal.cuh"

namespace fdtd {

struct AdjArgs {
    Geom g;
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
    float kr[3];                  // anisotropy factors of the pressure bracket (x, y, z)
    const float *nbr;             // density: -dtr / rho per node [vol], or null (rho = 1)
    const float *s_tape;          // bracket of this step [nshots][vol]
    const float *slab_tape[3];    // (g, psiv_old, h, psip_old) per slab node, or null
    float *gradK;                 // [nshots][vol]
    float *gprof;                 // [3][3][nmax] or null
    int nmax;
};

__device__ __forceinline__ int axis_coord(int d, int z, int y, int x) { return d == 0 ? x : (d == 1 ? y : z); }
__device__ __forceinline__ int axis_len(const Geom &g, int d) { return d == 0 ? g.nx : (d == 1 ? g.ny : g.nz); }

// lam_h_d at node (z, y, x) of one shot (0 outside the grid)
__device__ __forceinline__ float lam_h(const AdjArgs &A, int d, int z, int y, int x, const float *ap,
                                       const float *apsip_in)
{
    const Geom &g = A.g;
    if (x < 0 || x >= g.nx || y < 0 || y >= g.ny || z < 0 || z >= g.nz)
        return 0.f;
    const long long o = (long long)z * g.plane + (long long)y * g.nxp + x;
    const float q = A.kr[d] * ap[o];   // kr_d mu, mu = kdt lam_p
    const int k = axis_coord(d, z, y, x);
    if (in_slab(k, axis_len(g, d), g.lo[d], g.hi[d]))
        return A.ck[d][k] * q + A.ca[d][k] * (apsip_in[slab_index(g, d, z, y, x)] + q);
    return q;
}

__device__ __forceinline__ float lam_g(const AdjArgs &A, int d, int z, int y, int x, const float *av,
                                       const float *apsiv_in)
{
    const Geom &g = A.g;
    if (x < 0 || x >= g.nx || y < 0 || y >= g.ny || z < 0 || z >= g.nz)
        return 0.f;
    const long long o = (long long)z * g.plane + (long long)y * g.nxp + x;
    const float r = (A.nbr ? A.nbr[o] : -A.dtr) * av[o];
    const int k = axis_coord(d, z, y, x);
    if (in_slab(k, axis_len(g, d), g.lo[d], g.hi[d]))
        return A.ck[d][k] * r + A.ca[d][k] * (apsiv_in[slab_index(g, d, z, y, x)] + r);
    return r;
}

__global__ void adj_stage_a_kernel(AdjArgs A)
{
    const Geom &g = A.g;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z % g.nz, shot = blockIdx.z / g.nz;
    if (x >= g.nx || y >= g.ny)
        return;
    const long long fo = (long long)shot * g.vol;
    const long long o = (long long)z * g.plane + (long long)y * g.nxp + x;
    const float *ap = A.ap + fo;
    const float q = ap[o];   // mu = kdt lam_p
    A.gradK[fo + o] += -A.dt_over_vs * A.s_tape[fo + o] * (q / A.kdt[o]);
    const int dz[3] = {0, 0, 1}, dy[3] = {0, 1, 0}, dx[3] = {1, 0, 0};
    for (int d = 0; d < 3; ++d) {
        const float *psin = A.apsip_in[d] + (long long)shot * g.slab[d];
        float acc = 0.f;
#pragma unroll
        for (int l = 1; l <= 4; ++l)
            acc += A.c[l - 1] * (lam_h(A, d, z + l * dz[d], y + l * dy[d], x + l * dx[d], ap, psin) -
                                 lam_h(A, d, z - l * dz[d], y - l * dy[d], x - l * dx[d], ap, psin));
        A.av[d][fo + o] -= acc;
        const int k = axis_coord(d, z, y, x);
        if (in_slab(k, axis_len(g, d), g.lo[d], g.hi[d])) {
            const long long si = slab_index(g, d, z, y, x);
            const float qd = A.kr[d] * q;
            const float tot = psin[si] + qd;
            A.apsip_out[d][(long long)shot * g.slab[d] + si] = A.cb[d][k] * tot;
            if (A.gprof) {
                const float *tp = A.slab_tape[d] + ((long long)shot * g.slab[d] + si) * 4;
                atomicAdd(&A.gprof[(d * 3 + 0) * A.nmax + k], tot * tp[3]);
                atomicAdd(&A.gprof[(d * 3 + 1) * A.nmax + k], tot * tp[2]);
                atomicAdd(&A.gprof[(d * 3 + 2) * A.nmax + k], qd * tp[2]);
            }
        }
    }
}

__global__ void adj_stage_b_kernel(AdjArgs A)
{
    const Geom &g = A.g;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z % g.nz, shot = blockIdx.z / g.nz;
    if (x >= g.nx || y >= g.ny)
        return;
    const long long fo = (long long)shot * g.vol;
    const long long o = (long long)z * g.plane + (long long)y * g.nxp + x;
    const int dz[3] = {0, 0, 1}, dy[3] = {0, 1, 0}, dx[3] = {1, 0, 0};
    float acc = 0.f;
    for (int d = 0; d < 3; ++d) {
        const float *av = A.av[d] + fo;
        const float *psin = A.apsiv_in[d] + (long long)shot * g.slab[d];
#pragma unroll
        for (int l = 1; l <= 4; ++l)
            acc += A.c[l - 1] * (lam_g(A, d, z + l * dz[d], y + l * dy[d], x + l * dx[d], av, psin) -
                                 lam_g(A, d, z - l * dz[d], y - l * dy[d], x - l * dx[d], av, psin));
        const int k = axis_coord(d, z, y, x);
        if (in_slab(k, axis_len(g, d), g.lo[d], g.hi[d])) {
            const long long si = slab_index(g, d, z, y, x);
            const float r = (A.nbr ? A.nbr[o] : -A.dtr) * av[o];
            const float tot = psin[si] + r;
            A.apsiv_out[d][(long long)shot * g.slab[d] + si] = A.cb[d][k] * tot;
            if (A.gprof) {
                const float *tp = A.slab_tape[d] + ((long long)shot * g.slab[d] + si) * 4;
                atomicAdd(&A.gprof[(d * 3 + 0) * A.nmax + k], tot * tp[1]);
                atomicAdd(&A.gprof[(d * 3 + 1) * A.nmax + k], tot * tp[0]);
                atomicAdd(&A.gprof[(d * 3 + 2) * A.nmax + k], r * tp[0]);
            }
        }
    }
    A.ap[fo + o] -= A.kdt[o] * acc;
}

__global__ void adj_inject_kernel(float *ap, const float *kdt, Geom g, const int4 *rec, int nrec, int nshots,
                                  const float *resid, int nt_max, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrec * nshots)
        return;
    const int shot = i / nrec, k = i % nrec;
    const int4 q = rec[k];
    const float r = resid[((long long)shot * nt_max + n) * nrec + q.w];
    const long long o = (long long)q.x * g.plane + (long long)q.y * g.nxp + q.z;
    atomicAdd(&ap[(long long)shot * g.vol + o], kdt[o] * r);   // mu = kdt lam_p
}

// dJ/dc = 2 rho c dJ/dK with K = rho c^2 (rho fixed): -kdt vs / dt = K, and
// with a density rho = -dt vs / nbr (nbr = -dt vs / rho), else rho = 1.
__global__ void grad_vel_kernel(const float *gradK, const float *kdt, const float *nbr, Geom g, int nshots,
                                double vs_over_dt, double dt_vs, float *grad_vel)
{
    const long long n = (long long)g.nz * g.ny * g.nx;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx);
        const long long zy = i / g.nx;
        const long long o = zy * g.nxp + x;
        double acc = 0.0;
        for (int s = 0; s < nshots; ++s)
            acc += gradK[(long long)s * g.vol + o];
        const double K = -(double)kdt[o] * vs_over_dt;
        const double rho = nbr ? -dt_vs / (double)nbr[o] : 1.0;
        const double c = sqrt(K / rho);
        grad_vel[i] += (float)(2.0 * rho * c * acc);
    }
}

cudaError_t launch_adj_step(const fdtd_ctx *c, const AdjArgs &a)
{
    dim3 blk(32, 8);
    dim3 grid((c->g.nx + 31) / 32, (c->g.ny + 7) / 8, c->g.nz * c->d.nshots);
    adj_stage_a_kernel<<<grid, blk, 0, c->stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    // stage B reads the new lam_v and the incoming lam_psiv
    adj_stage_b_kernel<<<grid, blk, 0, c->stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adj_inject(const fdtd_ctx *c, const float *resid, int n)
{
    const int tot = c->nrec * c->d.nshots;
    if (tot == 0)
        return cudaSuccess;
    adj_inject_kernel<<<(tot + 255) / 256, 256, 0, c->stream>>>(c->ap, c->kdt, c->g, c->rec, c->nrec, c->d.nshots,
                                                                resid, c->d.nt_max, n);
    return cudaGetLastError();
}

cudaError_t launch_grad_vel(const fdtd_ctx *c, float *grad_vel)
{
    grad_vel_kernel<<<1216, 256, 0, c->stream>>>(c->gradK, c->kdt, c->var_rho ? c->nbr : nullptr, c->g,
                                                 c->d.nshots, c->vscale / c->d.dt, c->d.dt * c->vscale, grad_vel);
    return cudaGetLastError();
}

// One adjoint step on the current adjoint state (flips the memory-variable
// ping-pong).  s_tape / slab_tape: what the forward recompute taped for it.
cudaError_t adjoint_step(fdtd_ctx *c, const float *s_tape, float *const slab_tape[3], bool want_prof)
{
    AdjArgs a;
    a.g = c->g;
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
        a.slab_tape[d] = want_prof ? slab_tape[d] : nullptr;
    }
    for (int l = 0; l < 4; ++l)
        a.c[l] = (float)(kWeights[l] / c->d.h);
    a.dtr = (float)(c->d.dt * c->vscale);
    a.dt_over_vs = (float)(c->d.dt / c->vscale);
    for (int d = 0; d < 3; ++d)
        a.kr[d] = (float)c->kr[d];
    a.nbr = c->var_rho ? c->nbr : nullptr;
    a.s_tape = s_tape;
    a.gradK = c->gradK;
    a.gprof = want_prof ? c->gprof : nullptr;
    a.nmax = nmax;
    cudaError_t e = launch_adj_step(c, a);
    c->acur ^= 1;
    return e;
}
}  // namespace fdtd

// Auxiliary kernels of libfdtd: model set-up, field exchange between the
// caller's dense arrays and the internal (pitched / slab-compact, possibly
// 16-bit) layout, FP64 reductions, the learned-CPML coefficient map and its
// network (forward, backward, Adam).
#include <cmath>

#include "fdtd_internal.cuh"

namespace fdtd {

// ---------------------------------------------------------------------------
// model: kdt = -dt K / vscale with K = rho c^2 (rho = 1); min / max / invalid
// ---------------------------------------------------------------------------
// kdt = -dt rho c^2 / vscale (K = rho c^2) and, with a density, nbr = -dt
// vscale / rho, per node (0 in the row padding); rho = 1 without one.
__global__ void model_kernel(const float *__restrict__ vel, const float *__restrict__ rho, float *__restrict__ kdt,
                             float *__restrict__ nbr, Geom g, double dt, double vs, unsigned *minmax)
{
    unsigned vmin = 0x7f800000u, vmax = 0u, bad = 0u;
    // rows (z, y) across blocks, x across threads: no division per node
    for (long long zy = blockIdx.x; zy < (long long)g.nz * g.ny; zy += gridDim.x)
    for (int x = threadIdx.x; x < g.nxp; x += blockDim.x) {
        const long long i = zy * g.nxp + x;
        if (x >= g.nx) {
            kdt[i] = 0.f;
            if (rho)
                nbr[i] = 0.f;
            continue;
        }
        const float c = vel[zy * g.nx + x];
        const float r = rho ? rho[zy * g.nx + x] : 1.f;
        if (!(c > 0.f) || !isfinite(c) || !(r > 0.f) || !isfinite(r)) {
            bad++;
            kdt[i] = 0.f;
            if (rho)
                nbr[i] = 0.f;
            continue;
        }
        kdt[i] = (float)(-(dt / vs) * (double)r * (double)c * (double)c);
        if (rho)
            nbr[i] = (float)(-(dt * vs) / (double)r);
        const unsigned b = __float_as_uint(c);   // positive floats order like unsigned ints
        vmin = min(vmin, b);
        vmax = max(vmax, b);
    }
    atomicMin(&minmax[0], vmin);
    atomicMax(&minmax[1], vmax);
    if (bad)
        atomicAdd(&minmax[2], bad);
}

// ---------------------------------------------------------------------------
// local-velocity CPML grading: b, a of every node of the d-slab from the
// velocity c at that node, sigma_max(c) = -(q+1) c ln R / (2 L h) with the
// face's own L, sigma = sigma_max rho^q, kappa = 1 + (kmax - 1) rho^q,
// alpha = afrac sigma_max (1 - rho) at the node's normalised depth rho along
// d; written in the slab layout (the caller zeroes the padding first).
// ---------------------------------------------------------------------------
__global__ void local_coef_kernel(const float *__restrict__ vel, Geom g, int d, double h, double dt, double lnR,
                                  double kmax, double afrac, int q, float *__restrict__ lb, float *__restrict__ la,
                                  unsigned *bad)
{
    const int na = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
    const int lo = g.lo[d], hi = g.hi[d];
    unsigned nbad = 0;
    for (long long zy = blockIdx.x; zy < (long long)g.nz * g.ny; zy += gridDim.x)
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
        const long long i = zy * g.nx + x;
        const int z = (int)(zy / g.ny), y = (int)(zy - (long long)z * g.ny);
        const int j = d == 0 ? x : (d == 1 ? y : z);
        if (!in_slab(j, na, lo, hi))
            continue;
        const int L = j < lo ? lo : hi;
        const double rho = j < lo ? double(lo - j) / L : double(j - (na - 1 - hi)) / L;
        const double c = vel[i];
        double b = 0.0, a = 0.0;
        if (c > 0.0 && isfinite(c)) {
            const double smax = -(q + 1) * c * lnR / (2.0 * L * h);
            double rq = 1.0;
            for (int k = 0; k < q; ++k)
                rq *= rho;
            const double sigma = smax * rq, kappa = 1.0 + (kmax - 1.0) * rq, alpha = afrac * smax * (1.0 - rho);
            b = exp(-(sigma / kappa + alpha) * dt);
            const double den = kappa * (sigma + kappa * alpha);
            a = (sigma > 0.0 && den != 0.0) ? sigma * (b - 1.0) / den : 0.0;
        } else {
            nbad++;
        }
        const long long k = slab_index(g, d, z, y, x);
        lb[k] = (float)b;
        la[k] = (float)a;
    }
    if (nbad)
        atomicAdd(bad, nbad);
}

cudaError_t launch_local_coef(const fdtd_ctx *c, const float *vel, double R, double kmax, double afrac, int q)
{
    cudaError_t e = cudaMemsetAsync(c->minmax + 2, 0, 4, c->stream);
    for (int d = 0; d < 3 && e == cudaSuccess; ++d) {
        if (c->g.slab[d] == 0)
            continue;
        e = cudaMemsetAsync(c->lcoef[d][0], 0, (size_t)c->g.slab[d] * 4, c->stream);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(c->lcoef[d][1], 0, (size_t)c->g.slab[d] * 4, c->stream);
        if (e == cudaSuccess) {
            local_coef_kernel<<<1216, 256, 0, c->stream>>>(vel, c->g, d, c->d.h, c->d.dt, std::log(R), kmax, afrac, q,
                                                           c->lcoef[d][0], c->lcoef[d][1], c->minmax + 2);
            e = cudaGetLastError();
        }
    }
    return e;
}

cudaError_t launch_model(fdtd_ctx *c, const float *vel, const float *rho)
{
    const unsigned init[3] = {0x7f800000u, 0u, 0u};
    cudaError_t e = cudaMemcpyAsync(c->minmax, init, sizeof(init), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess)
        return e;
    model_kernel<<<1216, 256, 0, c->stream>>>(vel, rho, c->kdt, c->nbr, c->g, c->d.dt, c->vscale, c->minmax);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// field exchange.  kind 0: pitched [nz][ny][nxp]; kind 1..3: slab of axis
// kind-1.  Dense side: float [nz][ny][nx].
// ---------------------------------------------------------------------------
template <typename T>
__global__ void get_field_kernel(const T *__restrict__ src, float *__restrict__ dst, Geom g, int kind, float scale,
                                 const float *__restrict__ div)
{
    for (long long zy = blockIdx.x; zy < (long long)g.nz * g.ny; zy += gridDim.x)
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
        const long long i = zy * g.nx + x;
        const int z = (int)(zy / g.ny), y = (int)(zy - (long long)z * g.ny);
        float v = 0.f;
        if (kind == 0) {
            const long long o = (long long)z * g.plane + (long long)y * g.nxp + x;
            v = Io<T>::ld1(src + o);
            if (div)
                v /= div[o];
        } else {
            const int d = kind - 1;
            const int q = d == 0 ? x : (d == 1 ? y : z);
            const int nq = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
            if (in_slab(q, nq, g.lo[d], g.hi[d]))
                v = Io<T>::ld1(src + slab_index(g, d, z, y, x));
        }
        dst[i] = v * scale;
    }
}

template <typename T>
__global__ void set_field_kernel(T *__restrict__ dstf, const float *__restrict__ src, Geom g, int kind, float scale,
                                 const float *__restrict__ mul)
{
    for (long long zy = blockIdx.x; zy < (long long)g.nz * g.ny; zy += gridDim.x)
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
        const long long i = zy * g.nx + x;
        const int z = (int)(zy / g.ny), y = (int)(zy - (long long)z * g.ny);
        if (kind == 0) {
            const long long o = (long long)z * g.plane + (long long)y * g.nxp + x;
            Io<T>::st1(dstf + o, mul ? src[i] * scale * mul[o] : src[i] * scale);
        } else {
            const int d = kind - 1;
            const int q = d == 0 ? x : (d == 1 ? y : z);
            const int nq = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
            if (in_slab(q, nq, g.lo[d], g.hi[d]))
                Io<T>::st1(dstf + slab_index(g, d, z, y, x), src[i] * scale);
        }
    }
}

// `kscale` (or NULL): per-node factor of a full field, divided out on get and
// multiplied in on set (the adjoint pressure is stored as kdt lam_p)
cudaError_t launch_field(const fdtd_ctx *c, bool get, void *internal, float *dense, int kind, float scale,
                         bool is_f32, const float *kscale)
{
    const int blocks = 1216, threads = 256;
    if (is_f32 || c->d.storage == FDTD_F32) {
        if (get)
            get_field_kernel<float><<<blocks, threads, 0, c->stream>>>((const float *)internal, dense, c->g, kind,
                                                                        scale, kscale);
        else
            set_field_kernel<float><<<blocks, threads, 0, c->stream>>>((float *)internal, dense, c->g, kind, scale,
                                                                        kscale);
    } else if (c->d.storage == FDTD_F16) {
        if (get)
            get_field_kernel<__half><<<blocks, threads, 0, c->stream>>>((const __half *)internal, dense, c->g, kind,
                                                                         scale, nullptr);
        else
            set_field_kernel<__half><<<blocks, threads, 0, c->stream>>>((__half *)internal, dense, c->g, kind, scale,
                                                                         nullptr);
    } else {
        if (get)
            get_field_kernel<__nv_bfloat16><<<blocks, threads, 0, c->stream>>>((const __nv_bfloat16 *)internal,
                                                                                dense, c->g, kind, scale, nullptr);
        else
            set_field_kernel<__nv_bfloat16><<<blocks, threads, 0, c->stream>>>((__nv_bfloat16 *)internal, dense,
                                                                                c->g, kind, scale, nullptr);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 reductions: block partials into `part`, then one block sums them.
// ---------------------------------------------------------------------------
constexpr int RED_BLOCKS = 608;   // 4 x 152 SMs
constexpr int RED_THREADS = 256;

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double sh[RED_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0)
        sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = threadIdx.x < RED_THREADS / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1)
            r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;   // valid in thread 0
}

template <typename T>
__global__ void energy_kernel(const T *__restrict__ p, Geom g, int z0, int z1, int y0, int y1, int x0, int x1,
                              double *part)
{
    const int nyb = y1 - y0;
    double acc = 0.0;
    // rows of the box across blocks, x across threads
    for (long long r = blockIdx.x; r < (long long)(z1 - z0) * nyb; r += gridDim.x) {
        const int z = z0 + (int)(r / nyb), y = y0 + (int)(r % nyb);
        const T *row = p + (long long)z * g.plane + (long long)y * g.nxp;
        for (int x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
            const double v = Io<T>::ld1(row + x);
            acc += v * v;
        }
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0)
        part[blockIdx.x] = s;
}

__global__ void misfit_kernel(const float *__restrict__ tr, const float *__restrict__ dobs, float *resid,
                              long long nshots, long long nt, long long nt_max, long long nrec, double *part)
{
    const long long n = nshots * nt_max * nrec;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long step = (i / nrec) % nt_max;
        float r = 0.f;
        if (step < nt) {
            r = tr[i] - dobs[i];
            acc += (double)r * (double)r;
        }
        if (resid)
            resid[i] = r;
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0)
        part[blockIdx.x] = s;
}

__global__ void finish_sum_kernel(const double *part, int n, double scale, double *out)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        acc += part[i];
    const double s = block_sum(acc);
    if (threadIdx.x == 0)
        *out = s * scale;
}

cudaError_t launch_energy(const fdtd_ctx *c, const void *p, const int *box)
{
    switch (c->d.storage) {
    case FDTD_F16:
        energy_kernel<__half><<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>((const __half *)p, c->g, box[0], box[1],
                                                                          box[2], box[3], box[4], box[5], c->red);
        break;
    case FDTD_BF16:
        energy_kernel<__nv_bfloat16><<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>(
            (const __nv_bfloat16 *)p, c->g, box[0], box[1], box[2], box[3], box[4], box[5], c->red);
        break;
    default:
        energy_kernel<float><<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>((const float *)p, c->g, box[0], box[1],
                                                                         box[2], box[3], box[4], box[5], c->red);
    }
    finish_sum_kernel<<<1, RED_THREADS, 0, c->stream>>>(c->red, RED_BLOCKS, 1.0, c->red + RED_BLOCKS);
    return cudaGetLastError();
}

// Divergence check: sum of p^2 over every node of every shot (the energy
// reduction over a box whose z range runs through the shots, which follow
// each other in memory), then one thread raises ERR_NONFINITE if the sum is
// not finite or above `limit` (in stored units).
__global__ void divergence_flag_kernel(const double *sum, double limit, unsigned *err)
{
    const double s = *sum;
    if (!(s == s) || isinf(s) || s > limit)
        atomicOr(err, ERR_NONFINITE);
}

cudaError_t launch_divergence_check(const fdtd_ctx *c, double limit)
{
    const int box[6] = {0, c->g.nz * c->d.nshots, 0, c->g.ny, 0, c->g.nx};
    const cudaError_t e = launch_energy(c, c->p[c->cur], box);
    if (e != cudaSuccess)
        return e;
    divergence_flag_kernel<<<1, 1, 0, c->stream>>>(c->red + RED_BLOCKS, limit, c->err);
    return cudaGetLastError();
}

cudaError_t launch_misfit(const fdtd_ctx *c, const float *dobs, int nt, float *resid)
{
    misfit_kernel<<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>(c->traces, dobs, resid, c->d.nshots, nt, c->d.nt_max,
                                                             c->nrec, c->red);
    finish_sum_kernel<<<1, RED_THREADS, 0, c->stream>>>(c->red, RED_BLOCKS, 0.5, c->red + RED_BLOCKS);
    return cudaGetLastError();
}

// Misfit over a flat array of n values with `nblocks` partial sums written to
// `part` and the result to `*out` (both device memory the caller provides).
cudaError_t launch_misfit_flat(const float *tr, const float *dobs, float *resid, long long n, int nblocks,
                               double *part, double *out, cudaStream_t s)
{
    misfit_kernel<<<nblocks, RED_THREADS, 0, s>>>(tr, dobs, resid, 1, n, n, 1, part);
    finish_sum_kernel<<<1, RED_THREADS, 0, s>>>(part, nblocks, 0.5, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// learned CPML: per-cell (sigma, kappa, alpha) -> per-node (b, a, 1/kappa)
// and the chain rule back (Sec. 3.2 coefficient formulas, in double)
// ---------------------------------------------------------------------------
__device__ void ska_coefs(double s, double k, double al, double dt, double *b, double *a, double *kinv, double J[3][3])
{
    const double bb = exp(-(s / k + al) * dt);
    const double db[3] = {-dt / k * bb, dt * s / (k * k) * bb, -dt * bb};
    const double D = k * s + k * k * al;
    const double num = s * (bb - 1.0);
    const double dD[3] = {k, s + 2.0 * k * al, k * k};
    const double dnum[3] = {(bb - 1.0) + s * db[0], s * db[1], s * db[2]};
    *b = bb;
    *a = (s > 0.0 && D != 0.0) ? num / D : 0.0;
    *kinv = 1.0 / k;
    for (int m = 0; m < 3; ++m) {
        J[0][m] = db[m];
        J[1][m] = (s > 0.0 && D != 0.0) ? dnum[m] / D - num * dD[m] / (D * D) : 0.0;
        J[2][m] = 0.0;
    }
    J[2][1] = -1.0 / (k * k);
}

__global__ void ska_to_coef_kernel(const float *ska, int L, double dt, Geom g, float *coef, int nmax)
{
    const int j = threadIdx.x;
    if (j >= L)
        return;
    double b, a, kinv, J[3][3];
    ska_coefs(ska[3 * j], ska[3 * j + 1], ska[3 * j + 2], dt, &b, &a, &kinv, J);
    const int n[3] = {g.nx, g.ny, g.nz};
    for (int d = 0; d < 3; ++d) {
        const int nodes[2] = {j, n[d] - 1 - j};
        for (int s = 0; s < 2; ++s) {
            const int i = nodes[s];
            coef[(d * 3 + 0) * nmax + i] = (float)b;
            coef[(d * 3 + 1) * nmax + i] = (float)a;
            coef[(d * 3 + 2) * nmax + i] = (float)kinv;
        }
    }
}

__global__ void ska_backward_kernel(const float *ska, const float *gprof, int L, double dt, Geom g, int nmax,
                                    float *gska)
{
    const int j = threadIdx.x;
    if (j >= L)
        return;
    double b, a, kinv, J[3][3];
    ska_coefs(ska[3 * j], ska[3 * j + 1], ska[3 * j + 2], dt, &b, &a, &kinv, J);
    const int n[3] = {g.nx, g.ny, g.nz};
    double acc[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < 3; ++d) {
        const int nodes[2] = {j, n[d] - 1 - j};
        for (int s = 0; s < 2; ++s)
            for (int k = 0; k < 3; ++k) {
                const double gv = gprof[(d * 3 + k) * nmax + nodes[s]];
                for (int m = 0; m < 3; ++m)
                    acc[m] += gv * J[k][m];
            }
    }
    for (int m = 0; m < 3; ++m)
        gska[3 * j + m] = (float)acc[m];
}

cudaError_t launch_ska_to_coef(const fdtd_ctx *c, const float *ska, int L)
{
    const int nmax = max(c->g.nx, max(c->g.ny, c->g.nz));
    ska_to_coef_kernel<<<1, 64, 0, c->stream>>>(ska, L, c->d.dt, c->g, c->coef, nmax);
    return cudaGetLastError();
}

cudaError_t launch_ska_backward(const fdtd_ctx *c, const float *ska, const float *gprof, int L, float *gska)
{
    const int nmax = max(c->g.nx, max(c->g.ny, c->g.nz));
    ska_backward_kernel<<<1, 64, 0, c->stream>>>(ska, gprof, L, c->d.dt, c->g, nmax, gska);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// learned-CPML network 4 -> 64 -> 64 -> 3 (tanh), outputs through softplus
// ---------------------------------------------------------------------------
constexpr int H = 64;
constexpr int NPARAM = H * 4 + H + H * H + H + 3 * H + 3;   // 4675
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * 4, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + 3 * H;
constexpr int ACT = 2 * H + 3;
constexpr int MLP_BWD_MAX = 64;

__device__ __forceinline__ float softplus_f(float x) { return x > 20.f ? x : log1pf(expf(x)); }
__device__ __forceinline__ float sigmoid_f(float x) { return 1.f / (1.f + expf(-x)); }

__global__ void mlp_forward_kernel(const float *__restrict__ th, const float *__restrict__ X, int n, float ssc,
                                   float asc, float *out, float *act)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n)
        return;
    float h1[H], h2[H];
    for (int i = 0; i < H; ++i) {
        float z = th[OFF_B1 + i];
        for (int k = 0; k < 4; ++k)
            z += th[OFF_W1 + i * 4 + k] * X[4 * s + k];
        h1[i] = tanhf(z);
    }
    for (int i = 0; i < H; ++i) {
        float z = th[OFF_B2 + i];
        for (int k = 0; k < H; ++k)
            z += th[OFF_W2 + i * H + k] * h1[k];
        h2[i] = tanhf(z);
    }
    float o[3];
    for (int i = 0; i < 3; ++i) {
        float z = th[OFF_B3 + i];
        for (int k = 0; k < H; ++k)
            z += th[OFF_W3 + i * H + k] * h2[k];
        o[i] = z;
    }
    out[3 * s + 0] = ssc * softplus_f(o[0]);
    out[3 * s + 1] = 1.f + softplus_f(o[1]);
    out[3 * s + 2] = asc * softplus_f(o[2]);
    if (act) {
        float *a = act + (long long)s * ACT;
        for (int i = 0; i < H; ++i) {
            a[i] = h1[i];
            a[H + i] = h2[i];
        }
        for (int i = 0; i < 3; ++i)
            a[2 * H + i] = o[i];
    }
}

// One CTA: per-sample backpropagated signals into shared memory, then every
// parameter's gradient as a sum over samples (deterministic order).
__global__ void mlp_backward_kernel(const float *__restrict__ th, const float *__restrict__ X, int n,
                                    const float *__restrict__ act, const float *__restrict__ gout, float ssc,
                                    float asc, float *gth)
{
    __shared__ float go[MLP_BWD_MAX][3];
    __shared__ float gz2[MLP_BWD_MAX][H];
    __shared__ float gz1[MLP_BWD_MAX][H];
    const int tid = threadIdx.x;
    for (int idx = tid; idx < n * 3; idx += blockDim.x) {
        const int s = idx / 3, k = idx % 3;
        const float sc = k == 0 ? ssc : (k == 1 ? 1.f : asc);
        go[s][k] = gout[3 * s + k] * sc * sigmoid_f(act[(long long)s * ACT + 2 * H + k]);
    }
    __syncthreads();
    for (int idx = tid; idx < n * H; idx += blockDim.x) {
        const int s = idx / H, i = idx % H;
        float acc = 0.f;
        for (int k = 0; k < 3; ++k)
            acc += go[s][k] * th[OFF_W3 + k * H + i];
        const float h2 = act[(long long)s * ACT + H + i];
        gz2[s][i] = acc * (1.f - h2 * h2);
    }
    __syncthreads();
    for (int idx = tid; idx < n * H; idx += blockDim.x) {
        const int s = idx / H, j = idx % H;
        float acc = 0.f;
        for (int i = 0; i < H; ++i)
            acc += gz2[s][i] * th[OFF_W2 + i * H + j];
        const float h1 = act[(long long)s * ACT + j];
        gz1[s][j] = acc * (1.f - h1 * h1);
    }
    __syncthreads();
    for (int p = tid; p < NPARAM; p += blockDim.x) {
        float acc = 0.f;
        if (p < OFF_B1) {
            const int i = (p - OFF_W1) / 4, k = (p - OFF_W1) % 4;
            for (int s = 0; s < n; ++s)
                acc += gz1[s][i] * X[4 * s + k];
        } else if (p < OFF_W2) {
            const int i = p - OFF_B1;
            for (int s = 0; s < n; ++s)
                acc += gz1[s][i];
        } else if (p < OFF_B2) {
            const int i = (p - OFF_W2) / H, k = (p - OFF_W2) % H;
            for (int s = 0; s < n; ++s)
                acc += gz2[s][i] * act[(long long)s * ACT + k];
        } else if (p < OFF_W3) {
            const int i = p - OFF_B2;
            for (int s = 0; s < n; ++s)
                acc += gz2[s][i];
        } else if (p < OFF_B3) {
            const int i = (p - OFF_W3) / H, k = (p - OFF_W3) % H;
            for (int s = 0; s < n; ++s)
                acc += go[s][i] * act[(long long)s * ACT + H + k];
        } else {
            const int i = p - OFF_B3;
            for (int s = 0; s < n; ++s)
                acc += go[s][i];
        }
        gth[p] = acc;
    }
}

__global__ void adam_kernel(float *th, const float *g, float *m, float *v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

cudaError_t launch_mlp_forward(const float *th, const float *X, int n, float ssc, float asc, float *out, float *act,
                               cudaStream_t s)
{
    mlp_forward_kernel<<<(n + 63) / 64, 64, 0, s>>>(th, X, n, ssc, asc, out, act);
    return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const float *th, const float *X, int n, const float *act, const float *gout,
                                float ssc, float asc, float *gth, cudaStream_t s)
{
    mlp_backward_kernel<<<1, 256, 0, s>>>(th, X, n, act, gout, ssc, asc, gth);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *th, const float *g, float *m, float *v, int n, float lr, float b1, float b2, float eps,
                        float c1, float c2, cudaStream_t s)
{
    adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(th, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

// Gradient of the pre-fit loss of the learned grading,
//   loss = sum_j [((sigma_j - s*_j) / ss)^2 + (kappa_j - k*_j)^2 + ((alpha_j - a*_j) / as)^2],
// with respect to the network outputs (one block; the loss summed in double).
__global__ void fit_gradient_kernel(const float *out, const float *tgt, int n, float ssc, float asc, float *gout,
                                    float *loss)
{
    const double w[3] = {1.0 / ((double)ssc * ssc), 1.0, 1.0 / ((double)asc * asc)};
    double acc = 0.0;
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) {
        const double d = (double)out[i] - (double)tgt[i];
        gout[i] = (float)(2.0 * d * w[i % 3]);
        acc += d * d * w[i % 3];
    }
    const double sum = block_sum(acc);
    if (threadIdx.x == 0 && loss)
        *loss = (float)sum;
}

cudaError_t launch_fit_gradient(const float *out, const float *tgt, int n, float ssc, float asc, float *gout,
                                float *loss, cudaStream_t s)
{
    fit_gradient_kernel<<<1, RED_THREADS, 0, s>>>(out, tgt, n, ssc, asc, gout, loss);
    return cudaGetLastError();
}

int mlp_nparam() { return NPARAM; }
int mlp_bwd_max() { return MLP_BWD_MAX; }

}  // namespace fdtd

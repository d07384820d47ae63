// Host side of the libfdtd C ABI (declared in include/fdtd.h): argument
// validation, workspace layout, TMA descriptors, CPML profiles (paper
// Sec. 3.2, Tab. 2), receiver binning, time stepping with checkpoints, the
// checkpoint-and-recompute adjoint driver and the reductions.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "fdtd_internal.cuh"

namespace fdtd {
cudaError_t launch_step(const fdtd_ctx *c, const StepArgs &a, int set, cudaStream_t stream);
int step_occupancy(int storage, int *blocks);
cudaError_t launch_model(fdtd_ctx *c, const float *vel, const float *rho);
cudaError_t launch_field(const fdtd_ctx *c, bool get, void *internal, float *dense, int kind, float scale,
                         bool is_f32, const float *kscale);
cudaError_t launch_energy(const fdtd_ctx *c, const void *p, const int *box);
cudaError_t launch_misfit(const fdtd_ctx *c, const float *dobs, int nt, float *resid);
cudaError_t launch_divergence_check(const fdtd_ctx *c, double limit);
cudaError_t launch_ska_to_coef(const fdtd_ctx *c, const float *ska, int L);
cudaError_t launch_local_coef(const fdtd_ctx *c, const float *vel, double R, double kmax, double afrac, int q);
cudaError_t launch_ska_backward(const fdtd_ctx *c, const float *ska, const float *gprof, int L, float *gska);
cudaError_t launch_mlp_forward(const float *th, const float *X, int n, float ssc, float asc, float *out, float *act,
                               cudaStream_t s);
cudaError_t launch_mlp_backward(const float *th, const float *X, int n, const float *act, const float *gout,
                                float ssc, float asc, float *gth, cudaStream_t s);
cudaError_t launch_adam(float *th, const float *g, float *m, float *v, int n, float lr, float b1, float b2, float eps,
                        float c1, float c2, cudaStream_t s);
cudaError_t launch_fit_gradient(const float *out, const float *tgt, int n, float ssc, float asc, float *gout,
                                float *loss, cudaStream_t s);
cudaError_t launch_exchange(fdtd_ctx *dst, const fdtd_ctx *src, const int box[6], const int shift[3]);
cudaError_t launch_adj_inject(const fdtd_ctx *c, const float *resid, int n);
cudaError_t launch_grad_vel(const fdtd_ctx *c, float *grad_vel);
cudaError_t adjoint_step(fdtd_ctx *c, const float *s_tape, float *const slab_tape[3], bool want_prof);
cudaError_t adjoint_step_fused(fdtd_ctx *c, const float *s_tape);
int mlp_nparam();
int mlp_bwd_max();
}  // namespace fdtd

using namespace fdtd;

namespace {

int fail(fdtd_ctx *c, int status, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->last_error, sizeof(c->last_error), fmt, ap);
        va_end(ap);
    }
    return status;
}

#define CUDA_TRY(c, expr)                                                                          \
    do {                                                                                           \
        cudaError_t e_ = (expr);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail((c), FDTD_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));                 \
    } while (0)

size_t up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

struct Layout {
    Geom g;
    int es;
    int tiles_x, tiles_y;
    size_t p[2], v[3][2], psiv[3][2], psip[3];
    size_t kdt, nbr, coef, wav, src, rec, rec_off, err, red, minmax;
    int ncp;
    size_t ckpt, ckpt_slot, tape_s, tape_slab[3], ap[2], av[3][2], apsiv[3][2], apsip[3][2], gradK, gprof;
    size_t lcoef[3][2];
    size_t total;
};

int nmax_of(const Geom &g) { return std::max(g.nx, std::max(g.ny, g.nz)); }

const char *check_desc(const fdtd_desc *d)
{
    if (!d)
        return "desc is NULL";
    if (d->nx < 1 || d->ny < 1 || d->nz < 1)
        return "grid dimensions must be >= 1";
    if ((long long)d->nx * d->ny * d->nz > (1LL << 36))
        return "grid too large";
    if (!(d->h > 0.0) || !(d->dt > 0.0) || !std::isfinite(d->h) || !std::isfinite(d->dt))
        return "h and dt must be positive";
    const int n[3] = {d->nx, d->ny, d->nz};
    for (int a = 0; a < 3; ++a) {
        const int lo = d->cpml_cells[2 * a], hi = d->cpml_cells[2 * a + 1];
        if (lo < 0 || hi < 0 || lo + hi > n[a])
            return "CPML cells must be >= 0 and fit inside their axis";
        if (a == 0 && lo + hi > 0 && n[a] - lo - hi < 4)
            return "the x interior between CPML layers must be at least 4 nodes wide";
    }
    if (d->storage != FDTD_F32 && d->storage != FDTD_F16 && d->storage != FDTD_BF16)
        return "unknown storage";
    if (d->tblock_k != 1 && d->tblock_k != 2 && d->tblock_k != 4)
        return "tblock_k must be 1, 2 or 4";
    if (d->nt_max < 1)
        return "nt_max must be >= 1";
    if (d->nshots < 1 || d->nshots > 1024)
        return "nshots must be in [1, 1024]";
    if (d->nrec_max < 0)
        return "nrec_max must be >= 0";
    if (d->checkpoint_every < 0)
        return "checkpoint_every must be >= 0";
    if (d->cpml_grad && d->checkpoint_every <= 0)
        return "cpml_grad needs checkpoint_every > 0";
    return nullptr;
}

void make_layout(const fdtd_desc *d, Layout *L)
{
    Geom &g = L->g;
    g.nx = d->nx;
    g.ny = d->ny;
    g.nz = d->nz;
    g.nxp = (d->nx + 7) / 8 * 8;
    g.plane = (long long)g.ny * g.nxp;
    g.vol = (long long)g.nz * g.plane;
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = d->cpml_cells[2 * a];
        g.hi[a] = d->cpml_cells[2 * a + 1];
        g.w[a] = g.lo[a] + g.hi[a];
    }
    x_slab_layout(g.nx, g.lo[0], g.hi[0], &g.xhi, &g.w[0]);
    g.slab[0] = (long long)g.nz * g.ny * g.w[0];
    g.slab[1] = (long long)g.nz * g.w[1] * g.nxp;
    g.slab[2] = (long long)g.w[2] * g.ny * g.nxp;
    L->es = d->storage == FDTD_F32 ? 4 : 2;
    L->tiles_x = (g.nx + TX - 1) / TX;
    L->tiles_y = (g.ny + TY - 1) / TY;
    const size_t S = (size_t)d->nshots;
    const size_t fb = up(S * g.vol * L->es);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o += up(bytes);
        return r;
    };
    for (int s = 0; s < 2; ++s)
        L->p[s] = take(fb);
    for (int a = 0; a < 3; ++a)
        for (int s = 0; s < 2; ++s)
            L->v[a][s] = take(fb);
    for (int a = 0; a < 3; ++a) {
        for (int s = 0; s < 2; ++s)
            L->psiv[a][s] = take(S * g.slab[a] * L->es);
        L->psip[a] = take(S * g.slab[a] * L->es);
    }
    L->kdt = take((size_t)g.vol * 4);
    L->nbr = take((size_t)g.vol * 4);
    L->coef = take((size_t)18 * nmax_of(g) * 4);
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 2; ++k)
            L->lcoef[a][k] = d->cpml_local ? take((size_t)g.slab[a] * 4) : 0;
    L->wav = take(S * d->nt_max * 4);
    L->src = take(S * 3 * 4);
    L->rec = take((size_t)std::max(d->nrec_max, 1) * 16);
    L->rec_off = take(((size_t)L->tiles_x * L->tiles_y * g.nz + 1) * 4);
    L->err = take(16);
    L->red = take(8 * 1024);
    L->minmax = take(16);
    L->ncp = 0;
    if (d->checkpoint_every > 0) {
        const int C = d->checkpoint_every;
        L->ncp = (d->nt_max + C - 1) / C;
        size_t slot = 4 * fb;
        for (int a = 0; a < 3; ++a)
            slot += 2 * up(S * g.slab[a] * L->es);
        L->ckpt_slot = slot;
        L->ckpt = take(slot * L->ncp);
        L->tape_s = take((size_t)C * S * g.vol * 4);
        for (int a = 0; a < 3; ++a)
            L->tape_slab[a] = d->cpml_grad ? take((size_t)C * S * g.slab[a] * 16) : 0;
        for (int s = 0; s < 2; ++s) {
            L->ap[s] = take(S * g.vol * 4);
            for (int a = 0; a < 3; ++a)
                L->av[a][s] = take(S * g.vol * 4);
        }
        for (int a = 0; a < 3; ++a)
            for (int s = 0; s < 2; ++s) {
                L->apsiv[a][s] = take(S * g.slab[a] * 4);
                L->apsip[a][s] = take(S * g.slab[a] * 4);
            }
        L->gradK = take(S * g.vol * 4);
        L->gprof = take((size_t)9 * nmax_of(g) * 4);
    }
    L->total = o;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// Tiled tensor map over a pitched field; out-of-range boxes read zeros.
int make_map(fdtd_ctx *c, CUtensorMap *m, void *base, int rank, CUtensorMapDataType dtype, int es,
             const uint32_t *box)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn)
        return fail(c, FDTD_ECUDA, "cuTensorMapEncodeTiled unavailable");
    const Geom &g = c->g;
    cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)c->d.nshots};
    cuuint64_t strides[3] = {(cuuint64_t)g.nxp * es, (cuuint64_t)g.plane * es, (cuuint64_t)g.vol * es};
    cuuint32_t bx[4] = {box[0], box[1], box[2], box[3]};
    cuuint32_t es1[4] = {1, 1, 1, 1};
    CUresult r = fn(m, dtype, rank, base, dims, strides, bx, es1, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(c, FDTD_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return FDTD_OK;
}

int build_maps(fdtd_ctx *c)
{
    const CUtensorMapDataType dt = c->d.storage == FDTD_F32
                                       ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                       : (c->d.storage == FDTD_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                   : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    const uint32_t bP[4] = {TX + 16, TY + 16, 1, 1}, bQ[4] = {TX, TY, 1, 1}, bVX[4] = {TX + 16, TY, 1, 1},
                   bVY[4] = {TX, TY + 8, 1, 1};
    for (int s = 0; s < 2; ++s) {
        int st;
        if ((st = make_map(c, &c->maps[s][0], c->p[s], 4, dt, c->es, bP)) ||
            (st = make_map(c, &c->maps[s][1], c->p[s], 4, dt, c->es, bQ)) ||
            (st = make_map(c, &c->maps[s][2], c->v[0][s], 4, dt, c->es, bVX)) ||
            (st = make_map(c, &c->maps[s][3], c->v[1][s], 4, dt, c->es, bVY)) ||
            (st = make_map(c, &c->maps[s][4], c->v[2][s], 4, dt, c->es, bQ)))
            return st;
    }
    const uint32_t bK[4] = {TX, TY, 1, 1};
    int st = make_map(c, &c->mapK, c->kdt, 3, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, bK);
    if (st || c->ncp == 0)
        return st;
    const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const uint32_t b48[4] = {TX + 16, TY + 16, 1, 1}, bx[4] = {TX + 8, TY, 1, 1}, by[4] = {TX, TY + 8, 1, 1};
    for (int s = 0; s < 2; ++s)
        if ((st = make_map(c, &c->amaps[s][0], c->apb[s], 4, f32, 4, b48)) ||
            (st = make_map(c, &c->amaps[s][1], c->apb[s], 4, f32, 4, bQ)) ||
            (st = make_map(c, &c->amaps[s][2], c->avb[0][s], 4, f32, 4, bx)) ||
            (st = make_map(c, &c->amaps[s][3], c->avb[1][s], 4, f32, 4, by)) ||
            (st = make_map(c, &c->amaps[s][4], c->avb[2][s], 4, f32, 4, bQ)))
            return st;
    return FDTD_OK;
}

// Choose the z-chunk so that the grid fills the resident CTA slots evenly,
// counting the 8-plane prologue that each chunk re-reads.
void choose_zchunk(fdtd_ctx *c)
{
    int dev = 0, nsm = 152, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (step_occupancy(c->d.storage, &occ) != 0 || occ < 1)
        occ = 1;
    const long long slots = (long long)nsm * occ;
    const long long per_z = (long long)c->tiles_x * c->tiles_y * c->d.nshots;
    const int nz = c->g.nz;
    int best = 1;
    double best_eff = -1.0;
    for (int k = 1; k <= std::max(1, nz / 16); ++k) {
        const int zc = (nz + k - 1) / k;
        const int kk = (nz + zc - 1) / zc;
        const long long ctas = per_z * kk;
        const long long waves = (ctas + slots - 1) / slots;
        // time ~ waves x (planes + prologue); the 8 prologue iterations of a
        // chunk cost about a third of a full plane each
        const double eff = (double)nz * per_z / (double)slots / ((double)waves * (zc + 3.0));
        if (zc < 16 && k > 1)
            continue;
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = zc;
        }
    }
    // Large grids: chunks of about 48 planes (FP32); with 16-bit storage 96,
    // or 256 from 768 planes on.  CTAs that start together on chunks of
    // moderate length stay close in z, so the halo planes that neighbouring
    // tiles read are still in L2, while fewer chunk ends are re-read; at 512
    // planes the wave count decides between the longer chunks.  Measured with
    // the x-layer tiles launched first: FP32 1.049 ms at 512^3 against 1.069
    // with 32, 7.45 ms at 1024^3 against 7.66; FP16 6.97 ms at 1024^3 against
    // 7.16 with 96, and 1.021 ms at 512^3 against 1.092 with 256.
    int target = c->d.storage == FDTD_F32 ? 48 : (c->g.nz >= 768 ? 256 : 96);
    if (const char *e = getenv("FDTD_ZTARGET"))   // tuning: planes per middle chunk
        target = std::max(8, atoi(e));
    const int kt = (nz + target - 1) / target;
    const bool large = per_z * kt >= 2 * slots;
    if (large)
        best = (nz + kt - 1) / kt;
    c->zmid0 = 0;
    c->zmid1 = nz;
    const char *env = getenv("FDTD_ZCHUNK");
    if (env && atoi(env) > 0)
        best = std::min(atoi(env), nz);
    c->zchunk = best;
    c->nzchunks = (nz + best - 1) / best;
    c->zchunk_mid = best;
    // The fused adjoint's middle chunks: about 48 planes (measured on 256^3 x
    // 16 shots: 3.66 ms per adjoint step against 3.74 ms with 32 and 3.86
    // with 16); FDTD_AZTARGET overrides
    c->azchunk_target = 48;
    if (const char *e = getenv("FDTD_AZTARGET"))
        c->azchunk_target = std::max(8, atoi(e));
    // Forward steps on large grids: the planes that meet a z slab, with the
    // 4-plane reach of v_z, get a chunk of their own at each end, so that the
    // chunks in between run the step kernel's interior form.
    const int e1 = c->g.lo[2] + 4, e2 = nz - c->g.hi[2] - 4;
    if (large && !(env && atoi(env) > 0) && e2 - e1 >= target) {
        const int km = (e2 - e1 + target - 1) / target;
        c->zmid0 = e1;
        c->zmid1 = e2;
        c->zchunk_mid = (e2 - e1 + km - 1) / km;
    }
}

// Per-node CPML coefficients of one axis (normalised depth (L - j)/L at cell
// j of a face, j = 0 outermost).  half: the coefficients of the velocity
// nodes i + 1/2 of the staggered form, over the same slab index set: depth
// (lo - i - 1/2)/lo on the low face, (i + 1/2 - (n - 1 - hi))/hi, at most 1,
// on the high face.
// Polynomial grading of Sec. 3.2 / Tab. 2 at normalised depth rho of a face
// with L cells: sigma_max = -(q+1) c_ref ln R / (2 L h) (the continuous
// layer's normal-incidence round trip is then R), sigma = sigma_max rho^q,
// kappa = 1 + (kappa_max - 1) rho^q, alpha = alpha_frac sigma_max (1 - rho).
void grading_ska(double rho, int L, double h, double R, double kmax, double afrac, int q, double cref,
                 double *sigma, double *kappa, double *alpha)
{
    const double smax = -(q + 1) * cref * std::log(R) / (2.0 * L * h);
    const double rq = std::pow(rho, q);
    *sigma = smax * rq;
    *kappa = 1.0 + (kmax - 1.0) * rq;
    *alpha = afrac * smax * (1.0 - rho);
}

void host_profile(int n, int lo, int hi, double h, double dt, double R, double kmax, double afrac, int q, double cref,
                  bool half, float *b, float *a, float *kinv)
{
    for (int i = 0; i < n; ++i) {
        int L = 0;
        double rho = 0.0;
        if (i < lo) {
            L = lo;
            rho = double(lo - i) / lo;
        } else if (i >= n - hi) {
            L = hi;
            rho = double(i - (n - 1 - hi)) / hi;
        }
        if (L == 0) {
            b[i] = 0.f;
            a[i] = 0.f;
            kinv[i] = 1.f;
            continue;
        }
        if (half)   // the velocity node i + 1/2 (staggered form)
            rho = i < lo ? double(lo - i) - 0.5 : std::min(double(hi), double(i - (n - 1 - hi)) + 0.5);
        if (half)
            rho /= L;
        double sigma, kappa, alpha;
        grading_ska(rho, L, h, R, kmax, afrac, q, cref, &sigma, &kappa, &alpha);
        const double bb = std::exp(-(sigma / kappa + alpha) * dt);
        const double den = kappa * (sigma + kappa * alpha);
        b[i] = (float)bb;
        a[i] = (float)((sigma > 0.0 && den != 0.0) ? sigma * (bb - 1.0) / den : 0.0);
        kinv[i] = (float)(1.0 / kappa);
    }
}

// max over theta of 2 sum_l a_l sin(l theta): sampled, then refined
double symbol_max()
{
    double best = 0.0, bt = 0.0;
    const int N = 20000;
    for (int i = 0; i <= N; ++i) {
        const double th = M_PI * i / N;
        double s = 0.0;
        for (int l = 0; l < 4; ++l)
            s += 2.0 * kWeights[l] * std::sin((l + 1) * th);
        if (s > best) {
            best = s;
            bt = th;
        }
    }
    double lo = std::max(0.0, bt - M_PI / N), hi = std::min(M_PI, bt + M_PI / N);
    for (int it = 0; it < 200; ++it) {
        const double m1 = lo + (hi - lo) / 3, m2 = hi - (hi - lo) / 3;
        double s1 = 0, s2 = 0;
        for (int l = 0; l < 4; ++l) {
            s1 += 2.0 * kWeights[l] * std::sin((l + 1) * m1);
            s2 += 2.0 * kWeights[l] * std::sin((l + 1) * m2);
        }
        if (s1 < s2)
            lo = m1;
        else
            hi = m2;
    }
    double s = 0.0;
    for (int l = 0; l < 4; ++l)
        s += 2.0 * kWeights[l] * std::sin((l + 1) * 0.5 * (lo + hi));
    return std::max(best, s);
}

// c_max dt / h must not exceed 2 / (max_theta 2 sum_l a_l sin(l theta) * sqrt(sum_d kr_d))
// (3 axes, kr = 1: 2 / (sqrt(3) ...) = 0.6672).  The staggered symbol
// 2 sum_l c_l sin((l - 1/2) theta) peaks at theta = pi with 2 sum_l |c_l|
// (3 axes: 0.44884).
double stability_limit(const fdtd_ctx *c)
{
    double smax = symbol_max();
    if (c->staggered) {
        smax = 0.0;
        for (int l = 0; l < 4; ++l)
            smax += 2.0 * std::fabs(kStagWeights[l]);
    }
    return 2.0 / (std::sqrt(c->kr[0] + c->kr[1] + c->kr[2]) * smax);
}

bool fault_is(const char *what)
{
    const char *f = getenv("FDTD_FAULT");
    return f && strcmp(f, what) == 0;
}

// Streams and events of temporal blocking (tblock_k > 1).  The band height
// is 96 planes unless FDTD_TBAND says otherwise; it is never below 8, the
// dependence radius of one step along z.
int make_tblock(fdtd_ctx *c)
{
    const int k = c->d.tblock_k;
    if (k <= 1)
        return FDTD_OK;
    int band = 96;
    if (const char *e = getenv("FDTD_TBAND")) {
        const int v = atoi(e);
        if (v > 0)
            band = v;
    }
    c->tb_band = std::max(8, band);
    c->tb_nb = std::max(1, c->g.nz / c->tb_band);
    const size_t nev = (size_t)k * c->tb_nb;
    c->tb_ev = new (std::nothrow) cudaEvent_t[nev]();
    if (!c->tb_ev)
        return FDTD_ENOMEM;
    for (int s = 0; s < k; ++s)
        if (cudaStreamCreateWithFlags(&c->tb_stream[s], cudaStreamNonBlocking) != cudaSuccess)
            return FDTD_ECUDA;
    if (cudaEventCreateWithFlags(&c->tb_entry, cudaEventDisableTiming) != cudaSuccess)
        return FDTD_ECUDA;
    for (size_t i = 0; i < nev; ++i)
        if (cudaEventCreateWithFlags(&c->tb_ev[i], cudaEventDisableTiming) != cudaSuccess)
            return FDTD_ECUDA;
    return FDTD_OK;
}

// ---- kernel timing (fdtd_set_timing) ----
constexpr int kTimingPairs = 4096;

// Fold the recorded pairs of class k into the totals (waits for them).
cudaError_t timing_fold(fdtd_ctx *c, int k)
{
    for (int i = 0; i < c->tev_used[k]; ++i) {
        cudaError_t e = cudaEventSynchronize(c->tev[k][2 * i + 1]);
        if (e != cudaSuccess)
            return e;
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, c->tev[k][2 * i], c->tev[k][2 * i + 1]);
        if (e != cudaSuccess)
            return e;
        c->t_ms[k] += ms;
    }
    c->t_launch[k] += c->tev_used[k];
    c->tev_used[k] = 0;
    return cudaSuccess;
}

// Event before a launch of class k on `st` (no-op unless timing is on).
cudaError_t timing_begin(fdtd_ctx *c, int k, cudaStream_t st)
{
    if (!c->timing)
        return cudaSuccess;
    if (c->tev_used[k] == kTimingPairs) {
        const cudaError_t e = timing_fold(c, k);
        if (e != cudaSuccess)
            return e;
    }
    return cudaEventRecord(c->tev[k][2 * c->tev_used[k]], st);
}

// Event after that launch.
cudaError_t timing_end(fdtd_ctx *c, int k, cudaStream_t st)
{
    if (!c->timing)
        return cudaSuccess;
    const cudaError_t e = cudaEventRecord(c->tev[k][2 * c->tev_used[k] + 1], st);
    c->tev_used[k] += 1;
    return e;
}

void free_ctx(fdtd_ctx *c)
{
    for (int k = 0; k < 2; ++k)
        if (c->tev[k]) {
            for (int i = 0; i < 2 * kTimingPairs; ++i)
                if (c->tev[k][i])
                    cudaEventDestroy(c->tev[k][i]);
            delete[] c->tev[k];
        }
    if (c->tb_ev) {
        for (size_t i = 0; i < (size_t)c->d.tblock_k * c->tb_nb; ++i)
            if (c->tb_ev[i])
                cudaEventDestroy(c->tb_ev[i]);
        delete[] c->tb_ev;
    }
    if (c->tb_entry)
        cudaEventDestroy(c->tb_entry);
    for (int s = 0; s < 4; ++s)
        if (c->tb_stream[s])
            cudaStreamDestroy(c->tb_stream[s]);
    delete c;
}

StepArgs base_args(const fdtd_ctx *c)
{
    StepArgs a;
    memset(&a, 0, sizeof(a));
    a.g = c->g;
    a.tiles_x = c->tiles_x;
    a.tiles_y = c->tiles_y;
    x_layer_columns(c->g.nx, c->g.lo[0], c->g.hi[0], TX, &a.xcol_lo, &a.xcol_hi);
    a.zchunk = c->zchunk_mid;
    a.zbase = 0;
    a.zend = c->g.nz;
    a.zmid0 = c->zmid0;
    a.zmid1 = c->zmid1;
    const int nmax = nmax_of(c->g);
    for (int d = 0; d < 3; ++d) {
        a.cb[d] = c->coef + (d * 3 + 0) * nmax;
        a.ca[d] = c->coef + (d * 3 + 1) * nmax;
        a.ck[d] = c->coef + (d * 3 + 2) * nmax;
        const int hv = c->staggered ? 9 : 0;
        a.cbv[d] = c->coef + (hv + d * 3 + 0) * nmax;
        a.cav[d] = c->coef + (hv + d * 3 + 1) * nmax;
        a.ckv[d] = c->coef + (hv + d * 3 + 2) * nmax;
        a.psip[d] = c->psip[d];
    }
    for (int l = 0; l < 4; ++l)
        a.c[l] = (float)((c->staggered ? kStagWeights[l] : kWeights[l]) / c->d.h);
    for (int d = 0; d < 3; ++d) {
        a.lb[d] = c->cpml_local_set ? c->lcoef[d][0] : nullptr;
        a.la[d] = c->cpml_local_set ? c->lcoef[d][1] : nullptr;
    }
    // failure test (FDTD_FAULT=wait): one CTA's third stage gets no copies
    a.fault_it = fault_is("wait") ? 2 : -1;
    a.dtr = (float)(c->d.dt * c->vscale);   // rho = 1
    a.nbr = c->var_rho ? c->nbr : nullptr;
    a.sscale = c->sscale;
    for (int d = 0; d < 3; ++d)
        a.kr[d] = (float)c->kr[d];
    a.inv_sscale = 1.f / c->sscale;
    a.src = c->nt_w > 0 ? c->src : nullptr;
    a.wavelet = c->wavelet;
    a.nt_w = c->nt_w;
    a.rec_off = c->rec_off;
    a.rec = c->rec;
    a.nrec = c->nrec;
    a.nt_max = c->d.nt_max;
    a.traces = c->nrec > 0 ? c->traces : nullptr;
    a.err = c->err;
    return a;
}

bool needs_ckpt(const fdtd_ctx *c, int t)
{
    const int C = c->d.checkpoint_every;
    return C > 0 && t % C == 0 && t / C < c->ncp;
}

// m blocks of k = tblock_k steps.  The z range is cut into bands of at least
// 8 planes (the reach of one step along z).  Step s of a block runs on band b
// as soon as step s - 1 has finished bands b - 1, b and b + 1: each step has
// its own stream and waits on the event of band b + 1 of the step before
// (the previous block's last step, for s = 0).  Writes of step s land in the
// ping-pong set that step s - 2 wrote, whose readers (step s - 1 on bands
// b - 1 .. b + 1) are then done, so two sets suffice.  A band's intermediate
// state is read again soon after it is written, while it can still be held
// in L2.  Every node is computed exactly as by single steps.
int launch_blocks(fdtd_ctx *c, int m)
{
    const int k = c->d.tblock_k, nb = c->tb_nb;
    // planes per CTA within a band launch: the single-step chunk target (32
    // planes FP32, 96 16-bit), or FDTD_TBCHUNK.  Several chunks per band give
    // each launch more CTAs than one wave, so that the k streams' launches
    // backfill each other instead of starting together with a ragged tail.
    int tb_chunk = c->d.storage == FDTD_F32 ? 32 : 96;
    if (const char *e = getenv("FDTD_TBCHUNK"))
        if (atoi(e) > 0)
            tb_chunk = std::max(8, atoi(e));
    auto ev = [&](int s, int b) { return c->tb_ev[(size_t)s * nb + b]; };
    CUDA_TRY(c, cudaEventRecord(c->tb_entry, c->stream));
    for (int s = 0; s < k; ++s)
        CUDA_TRY(c, cudaStreamWaitEvent(c->tb_stream[s], c->tb_entry, 0));
    for (int blk = 0; blk < m; ++blk) {
        for (int dg = 0; dg < nb + k - 1; ++dg)
            for (int s = 0; s < k; ++s) {
                const int b = dg - s;
                if (b < 0 || b >= nb)
                    continue;
                cudaStream_t st = c->tb_stream[s];
                const int nxt = std::min(b + 1, nb - 1);
                if (s > 0)
                    CUDA_TRY(c, cudaStreamWaitEvent(st, ev(s - 1, nxt), 0));
                else if (blk > 0)
                    CUDA_TRY(c, cudaStreamWaitEvent(st, ev(k - 1, nxt), 0));
                StepArgs a = base_args(c);
                const int set = (c->cur + s) & 1;
                a.t = c->t + s;
                a.zbase = b * c->tb_band;
                a.zend = b == nb - 1 ? c->g.nz : (b + 1) * c->tb_band;
                // chunks of at most tb_chunk planes, equal within the band
                const int hb = a.zend - a.zbase, nch = (hb + tb_chunk - 1) / tb_chunk;
                a.zchunk = (hb + nch - 1) / nch;
                a.zmid0 = a.zbase;
                a.zmid1 = a.zend;
                a.p_in = c->p[set];
                a.p_out = c->p[set ^ 1];
                for (int d = 0; d < 3; ++d) {
                    a.v_in[d] = c->v[d][set];
                    a.v_out[d] = c->v[d][set ^ 1];
                    a.psiv_in[d] = c->psiv[d][set];
                    a.psiv_out[d] = c->psiv[d][set ^ 1];
                }
                CUDA_TRY(c, timing_begin(c, FDTD_TIMING_STEP, st));
                CUDA_TRY(c, launch_step(c, a, set, st));
                CUDA_TRY(c, timing_end(c, FDTD_TIMING_STEP, st));
                CUDA_TRY(c, cudaEventRecord(ev(s, b), st));
            }
        c->cur = (c->cur + k) & 1;
        c->t += k;
    }
    // the last step's final band comes after every other launch of the run
    CUDA_TRY(c, cudaStreamWaitEvent(c->stream, ev(k - 1, nb - 1), 0));
    return FDTD_OK;
}

int launch_one_step(fdtd_ctx *c, bool record, float *s_tape, float *const slab_tape[3])
{
    StepArgs a = base_args(c);
    a.t = c->t;
    const int s = c->cur;
    a.p_in = c->p[s];
    a.p_out = c->p[s ^ 1];
    for (int d = 0; d < 3; ++d) {
        a.v_in[d] = c->v[d][s];
        a.v_out[d] = c->v[d][s ^ 1];
        a.psiv_in[d] = c->psiv[d][s];
        a.psiv_out[d] = c->psiv[d][s ^ 1];
        a.slab_tape[d] = slab_tape ? slab_tape[d] : nullptr;
    }
    if (!record)
        a.traces = nullptr;
    a.s_tape = s_tape;
    CUDA_TRY(c, timing_begin(c, FDTD_TIMING_STEP, c->stream));
    CUDA_TRY(c, launch_step(c, a, s, c->stream));
    CUDA_TRY(c, timing_end(c, FDTD_TIMING_STEP, c->stream));
    c->cur ^= 1;
    c->t += 1;
    return FDTD_OK;
}

size_t field_bytes(const fdtd_ctx *c) { return (size_t)c->d.nshots * c->g.vol * c->es; }
size_t slab_bytes(const fdtd_ctx *c, int d) { return (size_t)c->d.nshots * c->g.slab[d] * c->es; }

int copy_state(fdtd_ctx *c, int slot, bool save)
{
    unsigned char *base = c->ckpt + (size_t)slot * c->ckpt_slot_bytes;
    size_t o = 0;
    const size_t fb = up(field_bytes(c));
    auto cp = [&](void *field, size_t bytes) -> cudaError_t {
        void *dst = save ? (void *)(base + o) : field;
        const void *src = save ? field : (const void *)(base + o);
        o += up(bytes);
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream) : cudaSuccess;
    };
    const int s = c->cur;
    CUDA_TRY(c, cp(c->p[s], field_bytes(c)));
    for (int d = 0; d < 3; ++d)
        CUDA_TRY(c, cp(c->v[d][s], field_bytes(c)));
    (void)fb;
    for (int d = 0; d < 3; ++d) {
        CUDA_TRY(c, cp(c->psiv[d][s], slab_bytes(c, d)));
        CUDA_TRY(c, cp(c->psip[d], slab_bytes(c, d)));
    }
    return FDTD_OK;
}

int memset_state(fdtd_ctx *c)
{
    for (int s = 0; s < 2; ++s) {
        CUDA_TRY(c, cudaMemsetAsync(c->p[s], 0, field_bytes(c), c->stream));
        for (int d = 0; d < 3; ++d) {
            CUDA_TRY(c, cudaMemsetAsync(c->v[d][s], 0, field_bytes(c), c->stream));
            if (slab_bytes(c, d))
                CUDA_TRY(c, cudaMemsetAsync(c->psiv[d][s], 0, slab_bytes(c, d), c->stream));
        }
    }
    for (int d = 0; d < 3; ++d)
        if (slab_bytes(c, d))
            CUDA_TRY(c, cudaMemsetAsync(c->psip[d], 0, slab_bytes(c, d), c->stream));
    if (c->ncp > 0) {
        const size_t fb = (size_t)c->d.nshots * c->g.vol * 4;
        c->aset = 0;
        c->ap = c->apb[0];
        for (int s = 0; s < 2; ++s)
            CUDA_TRY(c, cudaMemsetAsync(c->apb[s], 0, fb, c->stream));
        for (int d = 0; d < 3; ++d) {
            c->av[d] = c->avb[d][0];
            for (int s = 0; s < 2; ++s)
                CUDA_TRY(c, cudaMemsetAsync(c->avb[d][s], 0, fb, c->stream));
            const size_t sb = (size_t)c->d.nshots * c->g.slab[d] * 4;
            for (int s = 0; s < 2; ++s)
                if (sb) {
                    CUDA_TRY(c, cudaMemsetAsync(c->apsiv[d][s], 0, sb, c->stream));
                    CUDA_TRY(c, cudaMemsetAsync(c->apsip[d][s], 0, sb, c->stream));
                }
        }
    }
    CUDA_TRY(c, cudaMemsetAsync(c->err, 0, 16, c->stream));
    c->t = 0;
    c->cur = 0;
    c->acur = 0;
    return FDTD_OK;
}

bool needs_cpml(const fdtd_ctx *c)
{
    for (int i = 0; i < 6; ++i)
        if (c->d.cpml_cells[i] > 0)
            return true;
    return false;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int fdtd_abi_version(void) { return FDTD_ABI_VERSION; }

const char *fdtd_status_string(int s)
{
    switch (s) {
    case FDTD_OK:
        return "ok";
    case FDTD_EINVAL:
        return "invalid argument";
    case FDTD_ENOMEM:
        return "out of memory";
    case FDTD_ECUDA:
        return "CUDA error";
    case FDTD_ESTATE:
        return "call out of order";
    case FDTD_EUNSTABLE:
        return "unstable time step";
    case FDTD_EDIVERGED:
        return "non-finite values";
    case FDTD_ETIMEOUT:
        return "device wait timed out";
    case FDTD_EUNSUPPORTED:
        return "unsupported";
    default:
        return "unknown status";
    }
}

int fdtd_workspace_bytes(const fdtd_desc *desc, size_t *bytes)
{
    if (!bytes || check_desc(desc))
        return FDTD_EINVAL;
    if (desc->checkpoint_every > 0 && desc->storage != FDTD_F32)
        return FDTD_EUNSUPPORTED;
    Layout L;
    make_layout(desc, &L);
    *bytes = L.total;
    return FDTD_OK;
}

int fdtd_create(const fdtd_desc *desc, void *workspace, size_t workspace_bytes, fdtd_ctx **out)
{
    if (!out)
        return FDTD_EINVAL;
    *out = nullptr;
    if (fault_is("alloc"))
        return FDTD_ENOMEM;
    if (check_desc(desc))
        return FDTD_EINVAL;
    if (desc->checkpoint_every > 0 && desc->storage != FDTD_F32)
        return FDTD_EUNSUPPORTED;
    Layout L;
    make_layout(desc, &L);
    if (!workspace || workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255u))
        return FDTD_ENOMEM;
    fdtd_ctx *c = new (std::nothrow) fdtd_ctx;
    if (!c)
        return FDTD_ENOMEM;
    memset(c, 0, sizeof(*c));
    c->d = *desc;
    c->stream = (cudaStream_t)desc->stream;
    c->g = L.g;
    c->es = L.es;
    c->tiles_x = L.tiles_x;
    c->tiles_y = L.tiles_y;
    c->kr[0] = c->kr[1] = c->kr[2] = 1.0;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return FDTD_ECUDA;
    }
    c->vscale = 1.f;
    // FP16 keeps the whole state scaled by 2^10 (exact): small late-time
    // fields stay out of the FP16 subnormal range; the update is linear, so
    // only source, receivers, field exchange and the energy see the scale
    c->sscale = desc->storage == FDTD_F16 ? 1024.f : 1.f;
    c->ws = (unsigned char *)workspace;
    c->ws_bytes = workspace_bytes;
    unsigned char *w = c->ws;
    for (int s = 0; s < 2; ++s)
        c->p[s] = w + L.p[s];
    for (int d = 0; d < 3; ++d) {
        for (int s = 0; s < 2; ++s) {
            c->v[d][s] = w + L.v[d][s];
            c->psiv[d][s] = w + L.psiv[d][s];
        }
        c->psip[d] = w + L.psip[d];
    }
    c->kdt = (float *)(w + L.kdt);
    c->nbr = (float *)(w + L.nbr);
    c->coef = (float *)(w + L.coef);
    for (int d = 0; d < 3; ++d)
        for (int k = 0; k < 2; ++k)
            c->lcoef[d][k] = desc->cpml_local ? (float *)(w + L.lcoef[d][k]) : nullptr;
    c->wavelet = (float *)(w + L.wav);
    c->src = (int *)(w + L.src);
    c->rec = (int4 *)(w + L.rec);
    c->rec_off = (int *)(w + L.rec_off);
    c->err = (unsigned *)(w + L.err);
    c->red = (double *)(w + L.red);
    c->minmax = (unsigned *)(w + L.minmax);
    c->ncp = L.ncp;
    if (c->ncp > 0) {
        c->ckpt = w + L.ckpt;
        c->ckpt_slot_bytes = L.ckpt_slot;
        c->tape_s = (float *)(w + L.tape_s);
        for (int d = 0; d < 3; ++d) {
            c->tape_slab[d] = desc->cpml_grad ? (float *)(w + L.tape_slab[d]) : nullptr;
            for (int s = 0; s < 2; ++s)
                c->avb[d][s] = (float *)(w + L.av[d][s]);
            c->av[d] = c->avb[d][0];
            for (int s = 0; s < 2; ++s) {
                c->apsiv[d][s] = (float *)(w + L.apsiv[d][s]);
                c->apsip[d][s] = (float *)(w + L.apsip[d][s]);
            }
        }
        for (int s = 0; s < 2; ++s)
            c->apb[s] = (float *)(w + L.ap[s]);
        c->ap = c->apb[0];
        c->aset = 0;
        c->gradK = (float *)(w + L.gradK);
        c->gprof = (float *)(w + L.gprof);
    }
    int st;
    if ((st = build_maps(c)) != FDTD_OK) {
        delete c;
        return st;
    }
    choose_zchunk(c);
    // coefficient table: no CPML anywhere until set_cpml (b = a = 0, 1/kappa = 1)
    const int nmax = nmax_of(c->g);
    std::vector<float> coef((size_t)18 * nmax, 0.f);
    for (int d = 0; d < 6; ++d)
        for (int i = 0; i < nmax; ++i)
            coef[(d * 3 + 2) * nmax + i] = 1.f;
    cudaError_t e = cudaMemcpyAsync(c->coef, coef.data(), coef.size() * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->rec_off, 0, ((size_t)c->tiles_x * c->tiles_y * c->g.nz + 1) * 4, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess || memset_state(c) != FDTD_OK) {
        delete c;
        return FDTD_ECUDA;
    }
    if ((st = make_tblock(c)) != FDTD_OK) {
        free_ctx(c);
        return st;
    }
    *out = c;
    return FDTD_OK;
}

int fdtd_destroy(fdtd_ctx *c)
{
    if (!c)
        return FDTD_EINVAL;
    free_ctx(c);
    return FDTD_OK;
}

const char *fdtd_last_error(const fdtd_ctx *c) { return c ? c->last_error : "context is NULL"; }

int fdtd_set_model(fdtd_ctx *c, const float *vel, const float *rho)
{
    if (!c || !vel)
        return fail(c, FDTD_EINVAL, "vel is NULL");
    if (rho && c->staggered)
        return fail(c, FDTD_EUNSUPPORTED, "the staggered form is provided for constant density only");
    unsigned mm[3];
    c->vscale = 1.f;
    c->model_set = false;
    CUDA_TRY(c, launch_model(c, vel, rho));
    CUDA_TRY(c, cudaMemcpyAsync(mm, c->minmax, sizeof(mm), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (mm[2] != 0)
        return fail(c, FDTD_EINVAL, "%u nodes have a velocity or density that is not finite and positive", mm[2]);
    float vmin, vmax;
    memcpy(&vmin, &mm[0], 4);
    memcpy(&vmax, &mm[1], 4);
    const double limit = stability_limit(c);
    const double cfl = vmax * c->d.dt / c->d.h;
    if (cfl > limit)
        return fail(c, FDTD_EUNSTABLE, "c_max dt / h = %.6f exceeds the stability limit %.6f", cfl, limit);
    c->c_min = vmin;
    c->c_max = vmax;
    if (c->d.storage != FDTD_F32) {
        // impedance scaling keeps the stored velocities O(p) in 16-bit
        c->vscale = c->vscale_req > 0.f ? c->vscale_req : vmax;
        CUDA_TRY(c, launch_model(c, vel, rho));
    }
    c->var_rho = rho != nullptr;
    c->model_set = true;
    return FDTD_OK;
}

int fdtd_set_cpml(fdtd_ctx *c, double R, double kappa_max, double alpha_frac, int q, double c_ref)
{
    if (!c)
        return FDTD_EINVAL;
    if (!(R > 0.0 && R <= 1.0) || !(kappa_max >= 1.0) || !(alpha_frac >= 0.0) || q < 0)
        return fail(c, FDTD_EINVAL, "CPML parameters out of range");
    if (c_ref <= 0.0) {
        if (!c->model_set)
            return fail(c, FDTD_ESTATE, "c_ref <= 0 needs fdtd_set_model first");
        c_ref = c->c_max;
    }
    const int nmax = nmax_of(c->g);
    std::vector<float> coef((size_t)18 * nmax, 0.f);
    const int n[3] = {c->g.nx, c->g.ny, c->g.nz};
    for (int hv = 0; hv < 2; ++hv)
        for (int d = 0; d < 3; ++d) {
            float *t = &coef[(size_t)(9 * hv + d * 3) * nmax];
            host_profile(n[d], c->g.lo[d], c->g.hi[d], c->d.h, c->d.dt, R, kappa_max, alpha_frac, q, c_ref,
                         hv == 1, t, t + nmax, t + 2 * nmax);
        }
    CUDA_TRY(c, cudaMemcpyAsync(c->coef, coef.data(), coef.size() * 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->cpml_set = true;
    c->cpml_ska = false;
    c->cpml_local_set = false;
    return FDTD_OK;
}

int fdtd_set_anisotropy(fdtd_ctx *c, const double kr[3])
{
    if (!c || !kr)
        return fail(c, FDTD_EINVAL, "NULL argument");
    for (int d = 0; d < 3; ++d)
        if (!(kr[d] > 0.0) || !std::isfinite(kr[d]))
            return fail(c, FDTD_EINVAL, "anisotropy factors must be finite and positive");
    const double old[3] = {c->kr[0], c->kr[1], c->kr[2]};
    for (int d = 0; d < 3; ++d)
        c->kr[d] = kr[d];
    if (c->model_set) {
        const double cfl = c->c_max * c->d.dt / c->d.h, limit = stability_limit(c);
        if (cfl > limit) {
            for (int d = 0; d < 3; ++d)
                c->kr[d] = old[d];
            return fail(c, FDTD_EUNSTABLE, "c_max dt / h = %.6f exceeds the anisotropic limit %.6f", cfl, limit);
        }
    }
    return FDTD_OK;
}

int fdtd_set_cpml_local(fdtd_ctx *c, const float *vel, double R, double kappa_max, double alpha_frac, int q)
{
    if (!c || !vel)
        return fail(c, FDTD_EINVAL, "NULL argument");
    if (!c->d.cpml_local)
        return fail(c, FDTD_ESTATE, "the context was created without cpml_local");
    if (c->d.storage != FDTD_F32)
        return fail(c, FDTD_EUNSUPPORTED, "the local grading is provided for FP32 storage only");
    if (c->staggered)
        return fail(c, FDTD_EUNSUPPORTED, "the local grading is provided for the collocated form only");
    if (!c->model_set)
        return fail(c, FDTD_ESTATE, "fdtd_set_cpml_local needs fdtd_set_model first");
    // the 1D tables keep 1/kappa (and b, a graded with c_max for reference)
    int st = fdtd_set_cpml(c, R, kappa_max, alpha_frac, q, c->c_max);
    if (st != FDTD_OK)
        return st;
    unsigned bad = 0;
    CUDA_TRY(c, launch_local_coef(c, vel, R, kappa_max, alpha_frac, q));
    CUDA_TRY(c, cudaMemcpyAsync(&bad, c->minmax + 2, 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (bad)
        return fail(c, FDTD_EINVAL, "%u slab nodes have a velocity that is not finite and positive", bad);
    c->cpml_local_set = true;
    return FDTD_OK;
}

int fdtd_set_staggered(fdtd_ctx *c, int on)
{
    if (!c)
        return FDTD_EINVAL;
    if (on != 0 && on != 1)
        return fail(c, FDTD_EINVAL, "on must be 0 or 1");
    if (c->t != 0)
        return fail(c, FDTD_ESTATE, "the form is chosen before the first step (or after fdtd_reset)");
    if (on && c->d.storage != FDTD_F32)
        return fail(c, FDTD_EUNSUPPORTED, "the staggered form is provided for FP32 storage only");
    if (on && c->var_rho)
        return fail(c, FDTD_EUNSUPPORTED, "the staggered form is provided for constant density only");
    if (on && c->cpml_ska)
        return fail(c, FDTD_EUNSUPPORTED, "learned profiles are provided for the collocated form only");
    if (on && c->cpml_local_set)
        return fail(c, FDTD_EUNSUPPORTED, "the local grading is provided for the collocated form only");
    const bool old = c->staggered;
    c->staggered = on != 0;
    if (c->model_set) {
        const double cfl = c->c_max * c->d.dt / c->d.h, limit = stability_limit(c);
        if (cfl > limit) {
            c->staggered = old;
            return fail(c, FDTD_EUNSTABLE, "c_max dt / h = %.6f exceeds the limit %.6f of the form", cfl, limit);
        }
    }
    return FDTD_OK;
}

int fdtd_set_cpml_ska(fdtd_ctx *c, const float *ska)
{
    if (!c || !ska)
        return fail(c, FDTD_EINVAL, "ska is NULL");
    const int L = c->d.cpml_cells[0];
    for (int i = 1; i < 6; ++i)
        if (c->d.cpml_cells[i] != L)
            return fail(c, FDTD_EINVAL, "learned profiles need equal CPML cells on all faces");
    if (L < 1 || L > 64)
        return fail(c, FDTD_EINVAL, "learned layer must have 1..64 cells");
    if (c->staggered)
        return fail(c, FDTD_EUNSUPPORTED, "learned profiles are provided for the collocated form only");
    CUDA_TRY(c, launch_ska_to_coef(c, ska, L));
    c->cpml_set = true;
    c->cpml_ska = true;
    c->cpml_local_set = false;
    return FDTD_OK;
}

int fdtd_cpml_grading(int L, double h, double c_ref, double R, double kappa_max, double alpha_frac, int q,
                      double *ska)
{
    if (!ska || L < 1 || L > 1024 || !(h > 0.0) || !(c_ref > 0.0) || !(R > 0.0 && R <= 1.0) || !(kappa_max >= 1.0) ||
        !(alpha_frac >= 0.0) || q < 0)
        return FDTD_EINVAL;
    for (int j = 0; j < L; ++j)
        grading_ska(double(L - j) / L, L, h, R, kappa_max, alpha_frac, q, c_ref, &ska[3 * j], &ska[3 * j + 1],
                    &ska[3 * j + 2]);
    return FDTD_OK;
}

int fdtd_cpml_ska_backward(fdtd_ctx *c, const float *ska, const float *gprof, float *gska)
{
    if (!c || !ska || !gprof || !gska)
        return fail(c, FDTD_EINVAL, "NULL argument");
    const int L = c->d.cpml_cells[0];
    for (int i = 1; i < 6; ++i)
        if (c->d.cpml_cells[i] != L)
            return fail(c, FDTD_EINVAL, "learned profiles need equal CPML cells on all faces");
    if (L < 1 || L > 64)
        return fail(c, FDTD_EINVAL, "learned layer must have 1..64 cells");
    CUDA_TRY(c, launch_ska_backward(c, ska, gprof, L, gska));
    return FDTD_OK;
}

int fdtd_inject(fdtd_ctx *c, const int *src_zyx, const float *wavelet, int nt)
{
    if (!c || !src_zyx || !wavelet)
        return fail(c, FDTD_EINVAL, "NULL argument");
    if (nt < 0 || nt > c->d.nt_max)
        return fail(c, FDTD_EINVAL, "nt must be in [0, nt_max]");
    for (int s = 0; s < c->d.nshots; ++s) {
        const int z = src_zyx[3 * s], y = src_zyx[3 * s + 1], x = src_zyx[3 * s + 2];
        if (z < 0 || z >= c->g.nz || y < 0 || y >= c->g.ny || x < 0 || x >= c->g.nx)
            return fail(c, FDTD_EINVAL, "source %d outside the grid", s);
    }
    memcpy(c->src_host, src_zyx, sizeof(int) * 3 * c->d.nshots);
    CUDA_TRY(c, cudaMemcpyAsync(c->src, c->src_host, sizeof(int) * 3 * c->d.nshots, cudaMemcpyHostToDevice,
                                c->stream));
    if (nt > 0) {
        // [nshots][nt] packed -> [nshots][nt] with row stride nt (kernel reads shot * nt_w + t)
        CUDA_TRY(c, cudaMemcpyAsync(c->wavelet, wavelet, sizeof(float) * nt * c->d.nshots, cudaMemcpyDeviceToDevice,
                                    c->stream));
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->nt_w = nt;
    return FDTD_OK;
}

int fdtd_record(fdtd_ctx *c, const int *rec_zyx, int nrec, float *traces)
{
    if (!c)
        return FDTD_EINVAL;
    if (nrec < 0 || nrec > c->d.nrec_max)
        return fail(c, FDTD_EINVAL, "nrec must be in [0, nrec_max]");
    if (nrec > 0 && (!rec_zyx || !traces))
        return fail(c, FDTD_EINVAL, "NULL receivers or traces");
    const int ntiles = c->tiles_x * c->tiles_y;
    std::vector<int4> rv(nrec);
    std::vector<int> tile_of(nrec);
    for (int r = 0; r < nrec; ++r) {
        const int z = rec_zyx[3 * r], y = rec_zyx[3 * r + 1], x = rec_zyx[3 * r + 2];
        if (z < 0 || z >= c->g.nz || y < 0 || y >= c->g.ny || x < 0 || x >= c->g.nx)
            return fail(c, FDTD_EINVAL, "receiver %d outside the grid", r);
        rv[r] = make_int4(z, y, x, r);
        tile_of[r] = (y / TY) * c->tiles_x + x / TX;
    }
    std::vector<int> order(nrec);
    for (int r = 0; r < nrec; ++r)
        order[r] = r;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        if (tile_of[a] != tile_of[b])
            return tile_of[a] < tile_of[b];
        if (rv[a].x != rv[b].x)
            return rv[a].x < rv[b].x;
        if (rv[a].y != rv[b].y)
            return rv[a].y < rv[b].y;
        return rv[a].z < rv[b].z;
    });
    // ranges per (tile, plane): the kernel reads a plane's receivers together
    const int nz = c->g.nz;
    const size_t nbin = (size_t)ntiles * nz;
    std::vector<int4> sorted(std::max(nrec, 1));
    std::vector<int> off(nbin + 1, 0);
    for (int i = 0; i < nrec; ++i) {
        sorted[i] = rv[order[i]];
        off[(size_t)tile_of[order[i]] * nz + sorted[i].x + 1]++;
    }
    for (size_t b = 0; b < nbin; ++b)
        off[b + 1] += off[b];
    if (nrec > 0)
        CUDA_TRY(c, cudaMemcpyAsync(c->rec, sorted.data(), sizeof(int4) * nrec, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->rec_off, off.data(), sizeof(int) * (nbin + 1), cudaMemcpyHostToDevice,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->nrec = nrec;
    c->traces = traces;
    return FDTD_OK;
}

int fdtd_step_n(fdtd_ctx *c, int n)
{
    if (!c)
        return FDTD_EINVAL;
    if (n < 0)
        return fail(c, FDTD_EINVAL, "n must be >= 0");
    if (!c->model_set)
        return fail(c, FDTD_ESTATE, "fdtd_set_model has not been called");
    if (needs_cpml(c) && !c->cpml_set)
        return fail(c, FDTD_ESTATE, "fdtd_set_cpml has not been called");
    if (fault_is("launch"))
        return fail(c, FDTD_ECUDA, "injected launch failure (FDTD_FAULT=launch)");
    const int k = c->d.tblock_k;
    for (int i = 0; i < n;) {
        if (needs_ckpt(c, c->t)) {
            int st = copy_state(c, c->t / c->d.checkpoint_every, true);
            if (st)
                return st;
        }
        // as many whole blocks of k steps as fit before n and before the next
        // checkpoint; a checkpoint inside a block leaves that block to single steps
        int m = 0;
        if (k > 1)
            while (i + (m + 1) * k <= n) {
                const int t0 = c->t + m * k;
                bool inside = false;
                for (int j = 1; j < k; ++j)
                    inside = inside || needs_ckpt(c, t0 + j);
                if (inside)
                    break;
                ++m;
                if (needs_ckpt(c, t0 + k))
                    break;
            }
        int st;
        const int t_before = c->t;
        if (m > 0) {
            st = launch_blocks(c, m);
            i += m * k;
        } else {
            st = launch_one_step(c, true, nullptr, nullptr);
            ++i;
        }
        if (st)
            return st;
        // divergence check when a multiple of div_every was reached
        if (c->div_every > 0 && c->t / c->div_every > t_before / c->div_every)
            CUDA_TRY(c, launch_divergence_check(c, c->div_limit));
    }
    return FDTD_OK;
}

int fdtd_set_divergence_check(fdtd_ctx *c, int every, double limit)
{
    if (!c)
        return FDTD_EINVAL;
    if (every < 0 || std::isnan(limit))
        return fail(c, FDTD_EINVAL, "every must be >= 0 and limit a number");
    c->div_every = every;
    c->div_limit = limit > 0.0 ? limit * (double)c->sscale * (double)c->sscale : HUGE_VAL;
    return FDTD_OK;
}

int fdtd_adjoint_step_n(fdtd_ctx *c, int n, const float *resid, float *grad_vel, float *grad_cpml)
{
    if (!c)
        return FDTD_EINVAL;
    const int C = c->d.checkpoint_every;
    if (C <= 0 || c->ncp == 0)
        return fail(c, FDTD_ESTATE, "the adjoint needs checkpoint_every > 0 at create time");
    if (n != c->t || n > c->d.nt_max)
        return fail(c, FDTD_ESTATE, "n must equal the current time index (%d) and be <= nt_max", c->t);
    if (grad_cpml && !c->d.cpml_grad)
        return fail(c, FDTD_EINVAL, "grad_cpml needs cpml_grad at create time");
    if (c->staggered && grad_cpml)
        return fail(c, FDTD_EUNSUPPORTED, "the CPML-profile gradient is for the collocated form (node profiles)");
    if (c->cpml_local_set && grad_cpml)
        return fail(c, FDTD_EUNSUPPORTED, "the CPML-profile gradient is for the 1D grading (per axis and node)");
    const bool want_prof = grad_cpml != nullptr;
    const int nmax = nmax_of(c->g);
    CUDA_TRY(c, cudaMemsetAsync(c->gradK, 0, (size_t)c->d.nshots * c->g.vol * 4, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->gprof, 0, (size_t)9 * nmax * 4, c->stream));
    const int tend = c->t;
    for (int seg = (tend - 1) / C; seg >= 0 && tend > 0; --seg) {
        const int s0 = seg * C, s1 = std::min(s0 + C, tend);
        c->cur = 0;
        int st = copy_state(c, seg, false);
        if (st)
            return st;
        c->t = s0;
        for (int k = s0; k < s1; ++k) {
            float *slab[3];
            for (int d = 0; d < 3; ++d)
                slab[d] = c->tape_slab[d] ? c->tape_slab[d] + (size_t)(k - s0) * c->d.nshots * c->g.slab[d] * 4
                                          : nullptr;
            st = launch_one_step(c, false, c->tape_s + (size_t)(k - s0) * c->d.nshots * c->g.vol,
                                 want_prof ? slab : nullptr);
            if (st)
                return st;
        }
        for (int k = s1 - 1; k >= s0; --k) {
            if (resid)
                CUDA_TRY(c, launch_adj_inject(c, resid, k));
            float *slab[3];
            for (int d = 0; d < 3; ++d)
                slab[d] = c->tape_slab[d] ? c->tape_slab[d] + (size_t)(k - s0) * c->d.nshots * c->g.slab[d] * 4
                                          : nullptr;
            const float *sk = c->tape_s + (size_t)(k - s0) * c->d.nshots * c->g.vol;
            // the fused kernel carries no profile gradient; that path keeps the node-per-thread kernels
            CUDA_TRY(c, timing_begin(c, FDTD_TIMING_ADJOINT, c->stream));
            if (want_prof)
                CUDA_TRY(c, adjoint_step(c, sk, slab, true));
            else
                CUDA_TRY(c, adjoint_step_fused(c, sk));
            CUDA_TRY(c, timing_end(c, FDTD_TIMING_ADJOINT, c->stream));
        }
    }
    if (grad_vel)
        CUDA_TRY(c, launch_grad_vel(c, grad_vel));
    if (grad_cpml) {
        // grad_cpml += gprof (tiny: via a host round trip on the stream)
        std::vector<float> a((size_t)9 * nmax), b((size_t)9 * nmax);
        CUDA_TRY(c, cudaMemcpyAsync(a.data(), c->gprof, a.size() * 4, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(b.data(), grad_cpml, b.size() * 4, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        for (size_t i = 0; i < a.size(); ++i)
            b[i] += a[i];
        CUDA_TRY(c, cudaMemcpyAsync(grad_cpml, b.data(), b.size() * 4, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    c->t = tend;
    return FDTD_OK;
}

int fdtd_get_field(fdtd_ctx *c, int which, int shot, float *dst)
{
    if (!c || !dst)
        return fail(c, FDTD_EINVAL, "NULL argument");
    if (shot < 0 || shot >= c->d.nshots)
        return fail(c, FDTD_EINVAL, "shot out of range");
    if (which < 0 || which > FDTD_ADJ_PSIP_Z)
        return fail(c, FDTD_EINVAL, "unknown field");
    if (which >= FDTD_ADJ_P && c->ncp == 0)
        return fail(c, FDTD_ESTATE, "adjoint fields need checkpoint_every > 0");
    const long long fo = (long long)shot * c->g.vol;
    void *ptr = nullptr;
    int kind = 0;
    float scale = 1.f;
    bool f32 = false;
    const int s = c->cur;
    if (which == FDTD_P) {
        ptr = (unsigned char *)c->p[s] + fo * c->es;
    } else if (which <= FDTD_VZ) {
        ptr = (unsigned char *)c->v[which - FDTD_VX][s] + fo * c->es;
        scale = 1.f / c->vscale;
    } else if (which <= FDTD_PSIV_Z) {
        const int d = which - FDTD_PSIV_X;
        ptr = (unsigned char *)c->psiv[d][s] + (long long)shot * c->g.slab[d] * c->es;
        kind = d + 1;
    } else if (which <= FDTD_PSIP_Z) {
        const int d = which - FDTD_PSIP_X;
        ptr = (unsigned char *)c->psip[d] + (long long)shot * c->g.slab[d] * c->es;
        kind = d + 1;
        scale = 1.f / c->vscale;
    } else {
        f32 = true;
        if (which == FDTD_ADJ_P)
            ptr = c->ap + fo;
        else if (which <= FDTD_ADJ_VZ)
            ptr = c->av[which - FDTD_ADJ_VX] + fo;
        else if (which <= FDTD_ADJ_PSIV_Z) {
            const int d = which - FDTD_ADJ_PSIV_X;
            ptr = c->apsiv[d][c->acur] + (long long)shot * c->g.slab[d];
            kind = d + 1;
        } else {
            const int d = which - FDTD_ADJ_PSIP_X;
            ptr = c->apsip[d][c->acur] + (long long)shot * c->g.slab[d];
            kind = d + 1;
        }
    }
    if (!f32)
        scale /= c->sscale;
    if (kind > 0 && c->g.slab[kind - 1] == 0) {
        CUDA_TRY(c, cudaMemsetAsync(dst, 0, (size_t)c->g.nz * c->g.ny * c->g.nx * 4, c->stream));
        return FDTD_OK;
    }
    CUDA_TRY(c, launch_field(c, true, ptr, dst, kind, scale, f32, which == FDTD_ADJ_P ? c->kdt : nullptr));
    return FDTD_OK;
}

int fdtd_set_field(fdtd_ctx *c, int which, int shot, const float *src)
{
    if (!c || !src)
        return fail(c, FDTD_EINVAL, "NULL argument");
    if (shot < 0 || shot >= c->d.nshots)
        return fail(c, FDTD_EINVAL, "shot out of range");
    if (which < 0 || which > FDTD_ADJ_PSIP_Z)
        return fail(c, FDTD_EINVAL, "unknown field");
    if (which >= FDTD_ADJ_P && c->ncp == 0)
        return fail(c, FDTD_ESTATE, "adjoint fields need checkpoint_every > 0");
    const long long fo = (long long)shot * c->g.vol;
    void *ptr = nullptr;
    int kind = 0;
    float scale = 1.f;
    bool f32 = false;
    const int s = c->cur;
    if (which == FDTD_P) {
        ptr = (unsigned char *)c->p[s] + fo * c->es;
    } else if (which <= FDTD_VZ) {
        ptr = (unsigned char *)c->v[which - FDTD_VX][s] + fo * c->es;
        scale = c->vscale;
    } else if (which <= FDTD_PSIV_Z) {
        const int d = which - FDTD_PSIV_X;
        ptr = (unsigned char *)c->psiv[d][s] + (long long)shot * c->g.slab[d] * c->es;
        kind = d + 1;
    } else if (which <= FDTD_PSIP_Z) {
        const int d = which - FDTD_PSIP_X;
        ptr = (unsigned char *)c->psip[d] + (long long)shot * c->g.slab[d] * c->es;
        kind = d + 1;
        scale = c->vscale;
    } else {
        f32 = true;
        if (which == FDTD_ADJ_P)
            ptr = c->ap + fo;
        else if (which <= FDTD_ADJ_VZ)
            ptr = c->av[which - FDTD_ADJ_VX] + fo;
        else if (which <= FDTD_ADJ_PSIV_Z) {
            const int d = which - FDTD_ADJ_PSIV_X;
            ptr = c->apsiv[d][c->acur] + (long long)shot * c->g.slab[d];
            kind = d + 1;
        } else {
            const int d = which - FDTD_ADJ_PSIP_X;
            ptr = c->apsip[d][c->acur] + (long long)shot * c->g.slab[d];
            kind = d + 1;
        }
    }
    if (!f32)
        scale *= c->sscale;
    if (kind > 0 && c->g.slab[kind - 1] == 0)
        return FDTD_OK;
    CUDA_TRY(c, launch_field(c, false, ptr, const_cast<float *>(src), kind, scale, f32,
                             which == FDTD_ADJ_P ? c->kdt : nullptr));
    return FDTD_OK;
}

int fdtd_reset(fdtd_ctx *c)
{
    if (!c)
        return FDTD_EINVAL;
    return memset_state(c);
}

int fdtd_time(const fdtd_ctx *c, int *t)
{
    if (!c || !t)
        return FDTD_EINVAL;
    *t = c->t;
    return FDTD_OK;
}

int fdtd_set_time(fdtd_ctx *c, int t)
{
    if (!c)
        return FDTD_EINVAL;
    if (t < 0)
        return fail(c, FDTD_EINVAL, "time index must be >= 0");
    if (c->d.checkpoint_every > 0)
        return fail(c, FDTD_EUNSUPPORTED, "the time index of a context with checkpoints starts at 0");
    c->t = t;
    return FDTD_OK;
}

int fdtd_sync(fdtd_ctx *c)
{
    if (!c)
        return FDTD_EINVAL;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    unsigned err = 0;
    CUDA_TRY(c, cudaMemcpy(&err, c->err, 4, cudaMemcpyDeviceToHost));
    if (err & ERR_TIMEOUT)
        return fail(c, FDTD_ETIMEOUT, "a bounded device-side wait gave up");
    if (err & ERR_NONFINITE)
        return fail(c, FDTD_EDIVERGED, "the field diverged (non-finite values, or the energy above the check's limit)");
    return FDTD_OK;
}

int fdtd_set_timing(fdtd_ctx *c, int on)
{
    if (!c)
        return FDTD_EINVAL;
    if (on) {
        for (int k = 0; k < 2; ++k) {
            if (!c->tev[k]) {
                c->tev[k] = new (std::nothrow) cudaEvent_t[2 * kTimingPairs]();
                if (!c->tev[k])
                    return fail(c, FDTD_ENOMEM, "timing events: host allocation failed");
                for (int i = 0; i < 2 * kTimingPairs; ++i)
                    CUDA_TRY(c, cudaEventCreate(&c->tev[k][i]));
            }
            CUDA_TRY(c, timing_fold(c, k));
            c->t_ms[k] = 0.0;
            c->t_launch[k] = 0;
        }
    }
    c->timing = on != 0;
    return FDTD_OK;
}

int fdtd_timing(fdtd_ctx *c, int kernel_class, double *ms, long long *launches)
{
    if (!c)
        return FDTD_EINVAL;
    if (kernel_class < 0 || kernel_class > 1)
        return fail(c, FDTD_EINVAL, "unknown kernel class %d", kernel_class);
    if (c->tev[kernel_class])
        CUDA_TRY(c, timing_fold(c, kernel_class));
    if (ms)
        *ms = c->t_ms[kernel_class];
    if (launches)
        *launches = c->t_launch[kernel_class];
    return FDTD_OK;
}

int fdtd_set_velocity_scale(fdtd_ctx *c, double scale)
{
    if (!c)
        return FDTD_EINVAL;
    if (!(scale >= 0.0) || !std::isfinite(scale) || scale > 3.0e38)
        return fail(c, FDTD_EINVAL, "velocity scale must be finite and >= 0");
    c->vscale_req = (float)scale;
    return FDTD_OK;
}

int fdtd_exchange(fdtd_ctx *dst, const fdtd_ctx *src, const int box[6], const int shift[3])
{
    if (!dst || !src || !box || !shift)
        return dst ? fail(dst, FDTD_EINVAL, "NULL argument") : FDTD_EINVAL;
    if (dst == src)
        return fail(dst, FDTD_EINVAL, "source and destination are the same context");
    if (dst->d.storage != src->d.storage || dst->d.nshots != src->d.nshots || dst->staggered != src->staggered)
        return fail(dst, FDTD_EINVAL, "contexts differ in storage, shots or form");
    if (dst->device != src->device)
        return fail(dst, FDTD_EUNSUPPORTED, "contexts on different GPUs (devices %d and %d) need peer access, "
                                            "which this build does not set up", src->device, dst->device);
    if (dst->t != src->t)
        return fail(dst, FDTD_ESTATE, "contexts are at different time indices (%d, %d)", dst->t, src->t);
    if (dst->vscale != src->vscale || dst->sscale != src->sscale)
        return fail(dst, FDTD_EINVAL, "contexts store velocities at different scales (%g, %g): use "
                                      "fdtd_set_velocity_scale", (double)dst->vscale, (double)src->vscale);
    const int nd[3] = {dst->g.nz, dst->g.ny, dst->g.nx}, ns[3] = {src->g.nz, src->g.ny, src->g.nx};
    for (int a = 0; a < 3; ++a) {
        const int lo = box[2 * a], hi = box[2 * a + 1];
        if (lo > hi || lo < 0 || hi > nd[a] || lo + shift[a] < 0 || hi + shift[a] > ns[a])
            return fail(dst, FDTD_EINVAL, "box [%d, %d) + %d outside the grids on axis %c", lo, hi, shift[a], "zyx"[a]);
    }
    if (box[0] == box[1] || box[2] == box[3] || box[4] == box[5])
        return FDTD_OK;
    CUDA_TRY(dst, launch_exchange(dst, src, box, shift));
    return FDTD_OK;
}

int fdtd_energy(fdtd_ctx *c, int shot, const int box[6], double *out)
{
    if (!c || !box || !out)
        return fail(c, FDTD_EINVAL, "NULL argument");
    if (shot < 0 || shot >= c->d.nshots)
        return fail(c, FDTD_EINVAL, "shot out of range");
    if (box[0] < 0 || box[1] > c->g.nz || box[0] >= box[1] || box[2] < 0 || box[3] > c->g.ny || box[2] >= box[3] ||
        box[4] < 0 || box[5] > c->g.nx || box[4] >= box[5])
        return fail(c, FDTD_EINVAL, "box outside the grid or empty");
    const void *p = (const unsigned char *)c->p[c->cur] + (size_t)shot * c->g.vol * c->es;
    CUDA_TRY(c, launch_energy(c, p, box));
    CUDA_TRY(c, cudaMemcpyAsync(out, c->red + 608, 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    *out /= (double)c->sscale * (double)c->sscale;
    if (!std::isfinite(*out))
        return fail(c, FDTD_EDIVERGED, "non-finite energy");
    return FDTD_OK;
}

int fdtd_misfit(fdtd_ctx *c, const float *dobs, int nt, float *resid, double *out)
{
    if (!c || !dobs || !out)
        return fail(c, FDTD_EINVAL, "NULL argument");
    if (c->nrec == 0 || !c->traces)
        return fail(c, FDTD_ESTATE, "no receivers recorded");
    if (nt < 0 || nt > c->d.nt_max)
        return fail(c, FDTD_EINVAL, "nt must be in [0, nt_max]");
    CUDA_TRY(c, launch_misfit(c, dobs, nt, resid));
    CUDA_TRY(c, cudaMemcpyAsync(out, c->red + 608, 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (!std::isfinite(*out))
        return fail(c, FDTD_EDIVERGED, "non-finite misfit");
    return FDTD_OK;
}

int fdtd_mlp_forward(const float *theta, const float *X, int n, float sigma_scale, float alpha_scale, float *out,
                     float *act, void *stream)
{
    if (!theta || !X || !out || n < 1 || n > 1024)
        return FDTD_EINVAL;
    return launch_mlp_forward(theta, X, n, sigma_scale, alpha_scale, out, act, (cudaStream_t)stream) == cudaSuccess
               ? FDTD_OK
               : FDTD_ECUDA;
}

int fdtd_mlp_backward(const float *theta, const float *X, int n, const float *act, const float *gout,
                      float sigma_scale, float alpha_scale, float *gtheta, void *stream)
{
    if (!theta || !X || !act || !gout || !gtheta || n < 1 || n > mlp_bwd_max())
        return FDTD_EINVAL;
    return launch_mlp_backward(theta, X, n, act, gout, sigma_scale, alpha_scale, gtheta, (cudaStream_t)stream) ==
                   cudaSuccess
               ? FDTD_OK
               : FDTD_ECUDA;
}

int fdtd_adam_step(float *theta, const float *grad, float *m, float *v, int nparam, int t, float lr, float beta1,
                   float beta2, float eps, void *stream)
{
    if (!theta || !grad || !m || !v || nparam < 1 || t < 1)
        return FDTD_EINVAL;
    const float c1 = (float)(1.0 - std::pow((double)beta1, t));
    const float c2 = (float)(1.0 - std::pow((double)beta2, t));
    return launch_adam(theta, grad, m, v, nparam, lr, beta1, beta2, eps, c1, c2, (cudaStream_t)stream) == cudaSuccess
               ? FDTD_OK
               : FDTD_ECUDA;
}

int fdtd_mlp_fit_gradient(const float *out, const float *target, int n, float sigma_scale, float alpha_scale,
                          float *gout, float *loss, void *stream)
{
    if (!out || !target || !gout || n < 1 || n > 1024 || !(sigma_scale > 0.f) || !(alpha_scale > 0.f))
        return FDTD_EINVAL;
    return launch_fit_gradient(out, target, n, sigma_scale, alpha_scale, gout, loss, (cudaStream_t)stream) ==
                   cudaSuccess
               ? FDTD_OK
               : FDTD_ECUDA;
}

}  // extern "C"

// integrate.cu -- kick-drift-kick leapfrog with a shared timestep (Sec. 3.2 of
// Hirashima et al., SC'25), FP64 global diagnostics and field export.
//
// Velocities and internal energies are FP32; positions are advanced in FP64
// (Sec. 4.3).  The energy, momentum and angular momentum totals are FP64
// two-level reductions (block partials, then one block), so they do not
// depend on scheduling.
#include <utility>

#include "common.cuh"

namespace gnb {

__global__ void k_kick(PArr p, const float *__restrict__ ax, const float *__restrict__ ay,
                       const float *__restrict__ az, const float *__restrict__ dudt, int n, float hdt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    p.vx[i] = __fmaf_rn(ax[i], hdt, p.vx[i]);
    p.vy[i] = __fmaf_rn(ay[i], hdt, p.vy[i]);
    p.vz[i] = __fmaf_rn(az[i], hdt, p.vz[i]);
    if (p.type[i] == GNB_GAS) p.u[i] = __fmaf_rn(dudt[i], hdt, p.u[i]);
}

__global__ void k_drift(PArr p, int n, double dt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    p.x[i] = __dadd_rn(p.x[i], __dmul_rn((double)p.vx[i], dt));
    p.y[i] = __dadd_rn(p.y[i], __dmul_rn((double)p.vy[i], dt));
    p.z[i] = __dadd_rn(p.z[i], __dmul_rn((double)p.vz[i], dt));
}

// Predicted velocity and internal energy at the end of the step (used by
// the pressure and viscosity terms).
__global__ void k_predict(PArr p, const float *__restrict__ ax, const float *__restrict__ ay,
                          const float *__restrict__ az, const float *__restrict__ dudt, int n, float hdt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    p.vpx[i] = __fmaf_rn(ax[i], hdt, p.vx[i]);
    p.vpy[i] = __fmaf_rn(ay[i], hdt, p.vy[i]);
    p.vpz[i] = __fmaf_rn(az[i], hdt, p.vz[i]);
    p.up[i] = p.type[i] == GNB_GAS ? __fmaf_rn(dudt[i], hdt, p.u[i]) : 0.f;
}

// The first half of a KDK step in one pass: kick (k_kick), drift (k_drift)
// and the prediction (k_predict), with the same operations in the same
// order, so every result equals the three kernels' bit for bit; each
// particle's arrays are read and written once instead of three times.
__global__ void k_kick_drift_predict(PArr p, const float *__restrict__ ax, const float *__restrict__ ay,
                                     const float *__restrict__ az, const float *__restrict__ dudt, int n, float hdt,
                                     double dt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float a0 = ax[i], a1 = ay[i], a2 = az[i];
    const float vx = __fmaf_rn(a0, hdt, p.vx[i]), vy = __fmaf_rn(a1, hdt, p.vy[i]), vz = __fmaf_rn(a2, hdt, p.vz[i]);
    p.vx[i] = vx;
    p.vy[i] = vy;
    p.vz[i] = vz;
    p.x[i] = __dadd_rn(p.x[i], __dmul_rn((double)vx, dt));
    p.y[i] = __dadd_rn(p.y[i], __dmul_rn((double)vy, dt));
    p.z[i] = __dadd_rn(p.z[i], __dmul_rn((double)vz, dt));
    p.vpx[i] = __fmaf_rn(a0, hdt, vx);
    p.vpy[i] = __fmaf_rn(a1, hdt, vy);
    p.vpz[i] = __fmaf_rn(a2, hdt, vz);
    if (p.type[i] == GNB_GAS) {
        const float du = dudt[i];
        const float u = __fmaf_rn(du, hdt, p.u[i]);
        p.u[i] = u;
        p.up[i] = __fmaf_rn(du, hdt, u);
    } else {
        p.up[i] = 0.f;
    }
}

int kick_drift_predict(gnb_ctx *c, float hdt, double dt)
{
    int n = (int)c->n;
    gnb::counted(k_kick_drift_predict)<<<(n + 255) / 256, 256, 0, c->s>>>(c->P[c->cur], c->ax, c->ay, c->az,
                                                                           c->dudt, n, hdt, dt);
    GNB_LAUNCH_CHECK(c, "kick, drift, predict");
    return GNB_OK;
}

int kick(gnb_ctx *c, float hdt, bool)
{
    int n = (int)c->n;
    gnb::counted(k_kick)<<<(n + 255) / 256, 256, 0, c->s>>>(c->P[c->cur], c->ax, c->ay, c->az, c->dudt, n, hdt);
    GNB_LAUNCH_CHECK(c, "kick");
    return GNB_OK;
}

int drift(gnb_ctx *c, double dt)
{
    int n = (int)c->n;
    gnb::counted(k_drift)<<<(n + 255) / 256, 256, 0, c->s>>>(c->P[c->cur], n, dt);
    GNB_LAUNCH_CHECK(c, "drift");
    return GNB_OK;
}

int predict(gnb_ctx *c, float hdt)
{
    int n = (int)c->n;
    gnb::counted(k_predict)<<<(n + 255) / 256, 256, 0, c->s>>>(c->P[c->cur], c->ax, c->ay, c->az, c->dudt, n, hdt);
    GNB_LAUNCH_CHECK(c, "predict");
    return GNB_OK;
}

// total = external (already in a) + self-gravity; du/dt reset
__global__ void k_combine(int n, const float *__restrict__ gax, const float *__restrict__ gay,
                          const float *__restrict__ gaz, float *__restrict__ ax, float *__restrict__ ay,
                          float *__restrict__ az, float *__restrict__ dudt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    ax[i] += gax[i];
    ay[i] += gay[i];
    az[i] += gaz[i];
    dudt[i] = 0.f;
}

int zero_forces(gnb_ctx *c)
{
    int n = (int)c->n;
    gnb::counted(k_combine)<<<(n + 255) / 256, 256, 0, c->s>>>(n, c->gax, c->gay, c->gaz, c->ax, c->ay, c->az, c->dudt);
    GNB_LAUNCH_CHECK(c, "combine");
    return GNB_OK;
}

// ---------------------------------------------------------------- diagnostics
#define DG_BLOCKS 256
__global__ void k_diag_partial(PArr p, const float *__restrict__ pot, const float *__restrict__ pext, int n,
                               double *__restrict__ part)
{
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double m = p.m[i];
        double vx = p.vx[i], vy = p.vy[i], vz = p.vz[i];
        double x = p.x[i], y = p.y[i], z = p.z[i];
        acc[0] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        acc[1] += 0.5 * m * (double)pot[i];
        acc[2] += m * (double)pext[i];
        if (p.type[i] == GNB_GAS) acc[3] += m * (double)p.u[i];
        acc[4] += m * vx;
        acc[5] += m * vy;
        acc[6] += m * vz;
        acc[7] += m * (y * vz - z * vy);
        acc[8] += m * (z * vx - x * vz);
        acc[9] += m * (x * vy - y * vx);
    }
    __shared__ double sh[10][8];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 10; k++) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[k][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        double s = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) s += sh[threadIdx.x][q];
        part[blockIdx.x * 10 + threadIdx.x] = s;
    }
}

__global__ void k_diag_final(const double *__restrict__ part, int nb, double *__restrict__ out)
{
    int k = threadIdx.x;
    if (k >= 10) return;
    double s = 0;
    for (int b = 0; b < nb; b++) s += part[b * 10 + k];
    out[k] = s;
}

int diagnostics(gnb_ctx *c, double out[10])
{
    int n = (int)c->n;
    gnb::counted(k_diag_partial)<<<DG_BLOCKS, 256, 0, c->s>>>(c->P[c->cur], c->pot, c->pext, n, c->red_d);
    gnb::counted(k_diag_final)<<<1, 32, 0, c->s>>>(c->red_d, DG_BLOCKS, c->red_d + DG_BLOCKS * 10);
    GNB_LAUNCH_CHECK(c, "diagnostics");
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(out, c->red_d + DG_BLOCKS * 10, 10 * sizeof(double),
                                          cudaMemcpyDeviceToHost, c->s), "diagnostics copy"));
    return cuda_check(c, cudaStreamSynchronize(c->s), "diagnostics sync");
}

// ---------------------------------------------------------------- export
template <class T>
__global__ void k_scatter_orig(const T *__restrict__ src, const int *__restrict__ orig, int n, T *__restrict__ dst)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[orig[i]] = src[i];
}

__global__ void k_scatter_orig_zero_star(const float *__restrict__ src, const int *__restrict__ orig,
                                         const uint8_t *__restrict__ type, int n, float *__restrict__ dst)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[orig[i]] = type[i] == GNB_GAS ? src[i] : 0.f;
}

__global__ void k_scatter_orig_zero_star_d(const double *__restrict__ src, const int *__restrict__ orig,
                                           const uint8_t *__restrict__ type, int n, double *__restrict__ dst)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[orig[i]] = type[i] == GNB_GAS ? src[i] : 0.0;
}

__global__ void k_order_out(const int *__restrict__ orig, int n, int64_t *__restrict__ dst)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = orig[i];
}

__global__ void k_nodes_out(int4 *__restrict__ na, const uint64_t *__restrict__ skey, int nn,
                            int64_t *__restrict__ dst)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nn) return;
    int4 a = na[k];
    int lev = a.w & 255;
    dst[4 * k + 0] = lev;
    dst[4 * k + 1] = lev == 0 ? 0 : (int64_t)(skey[a.x] >> (3 * (GNB_MAXLEV - lev)));
    dst[4 * k + 2] = a.x;
    dst[4 * k + 3] = a.y;
}

__global__ void k_links_out(const int4 *__restrict__ na, const int4 *__restrict__ nb, int nn,
                            int64_t *__restrict__ dst)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nn) return;
    const int4 a = na[k];
    dst[3 * k + 0] = a.z;
    dst[3 * k + 1] = a.w >> 8;
    dst[3 * k + 2] = nb[k].w;
}

__global__ void k_groups_out(const int *__restrict__ groups, int ng, int64_t *__restrict__ dst)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < ng) dst[k] = groups[k];
}

// neighbour rows: row = gas rank of particle, entries = caller indices, ascending
__global__ void k_nbr_out(int ng, const int *__restrict__ nbr, const int *__restrict__ gslot,
                          const int *__restrict__ orig, const int *__restrict__ ggrank, int64_t *__restrict__ dst)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ng) return;
    int64_t v[64];
    for (int q = 0; q < 64; q++) v[q] = orig[gslot[nbr[(size_t)k * 64 + q]]];
    for (int a = 1; a < 64; a++) {
        int64_t t = v[a];
        int b = a - 1;
        while (b >= 0 && v[b] > t) { v[b + 1] = v[b]; b--; }
        v[b + 1] = t;
    }
    int64_t *row = dst + (size_t)ggrank[k] * 64;
    for (int q = 0; q < 64; q++) row[q] = v[q];
}

int scatter_out(gnb_ctx *c, int field, void *dst)
{
    int n = (int)c->n;
    int nb = (n + 255) / 256;
    PArr &a = c->P[c->cur];
    switch (field) {
    case GNB_F_X: gnb::counted(k_scatter_orig<double>)<<<nb, 256, 0, c->s>>>(a.x, a.orig, n, (double *)dst); break;
    case GNB_F_Y: gnb::counted(k_scatter_orig<double>)<<<nb, 256, 0, c->s>>>(a.y, a.orig, n, (double *)dst); break;
    case GNB_F_Z: gnb::counted(k_scatter_orig<double>)<<<nb, 256, 0, c->s>>>(a.z, a.orig, n, (double *)dst); break;
    case GNB_F_VX: gnb::counted(k_scatter_orig<float>)<<<nb, 256, 0, c->s>>>(a.vx, a.orig, n, (float *)dst); break;
    case GNB_F_VY: gnb::counted(k_scatter_orig<float>)<<<nb, 256, 0, c->s>>>(a.vy, a.orig, n, (float *)dst); break;
    case GNB_F_VZ: gnb::counted(k_scatter_orig<float>)<<<nb, 256, 0, c->s>>>(a.vz, a.orig, n, (float *)dst); break;
    case GNB_F_AX: gnb::counted(k_scatter_orig<float>)<<<nb, 256, 0, c->s>>>(c->ax, a.orig, n, (float *)dst); break;
    case GNB_F_AY: gnb::counted(k_scatter_orig<float>)<<<nb, 256, 0, c->s>>>(c->ay, a.orig, n, (float *)dst); break;
    case GNB_F_AZ: gnb::counted(k_scatter_orig<float>)<<<nb, 256, 0, c->s>>>(c->az, a.orig, n, (float *)dst); break;
    case GNB_F_AGRAV_X: gnb::counted(k_scatter_orig<float>)<<<nb, 256, 0, c->s>>>(c->gax, a.orig, n, (float *)dst); break;
    case GNB_F_AGRAV_Y: gnb::counted(k_scatter_orig<float>)<<<nb, 256, 0, c->s>>>(c->gay, a.orig, n, (float *)dst); break;
    case GNB_F_AGRAV_Z: gnb::counted(k_scatter_orig<float>)<<<nb, 256, 0, c->s>>>(c->gaz, a.orig, n, (float *)dst); break;
    case GNB_F_POT: gnb::counted(k_scatter_orig<float>)<<<nb, 256, 0, c->s>>>(c->pot, a.orig, n, (float *)dst); break;
    case GNB_F_POT_EXT: gnb::counted(k_scatter_orig<float>)<<<nb, 256, 0, c->s>>>(c->pext, a.orig, n, (float *)dst); break;
    case GNB_F_U: gnb::counted(k_scatter_orig_zero_star)<<<nb, 256, 0, c->s>>>(a.u, a.orig, a.type, n, (float *)dst); break;
    case GNB_F_DUDT:
        gnb::counted(k_scatter_orig_zero_star)<<<nb, 256, 0, c->s>>>(c->dudt, a.orig, a.type, n, (float *)dst);
        break;
    case GNB_F_RHO: gnb::counted(k_scatter_orig_zero_star)<<<nb, 256, 0, c->s>>>(c->rho, a.orig, a.type, n, (float *)dst); break;
    case GNB_F_PRES:
        gnb::counted(k_scatter_orig_zero_star)<<<nb, 256, 0, c->s>>>(c->pres, a.orig, a.type, n, (float *)dst);
        break;
    case GNB_F_CS: gnb::counted(k_scatter_orig_zero_star)<<<nb, 256, 0, c->s>>>(c->cs, a.orig, a.type, n, (float *)dst); break;
    case GNB_F_H2: gnb::counted(k_scatter_orig_zero_star_d)<<<nb, 256, 0, c->s>>>(a.h2, a.orig, a.type, n, (double *)dst); break;
    case GNB_F_KEY: gnb::counted(k_scatter_orig<uint64_t>)<<<nb, 256, 0, c->s>>>(c->skey, a.orig, n, (uint64_t *)dst); break;
    case GNB_F_LEVEL: gnb::counted(k_scatter_orig<int>)<<<nb, 256, 0, c->s>>>(c->hlev[0], a.orig, n, (int *)dst); break;
    case GNB_F_ID: gnb::counted(k_scatter_orig<int64_t>)<<<nb, 256, 0, c->s>>>(a.id, a.orig, n, (int64_t *)dst); break;
    case GNB_F_ORDER: gnb::counted(k_order_out)<<<nb, 256, 0, c->s>>>(a.orig, n, (int64_t *)dst); break;
    case GNB_F_NODES:
        gnb::counted(k_nodes_out)<<<(c->t.nnodes + 255) / 256, 256, 0, c->s>>>(c->t.na, c->skey, c->t.nnodes, (int64_t *)dst);
        break;
    case GNB_F_NODE_LINKS:
        gnb::counted(k_links_out)<<<(c->t.nnodes + 255) / 256, 256, 0, c->s>>>(c->t.na, c->t.nb, c->t.nnodes,
                                                                                  (int64_t *)dst);
        break;
    case GNB_F_GROUPS:
        gnb::counted(k_groups_out)<<<(c->t.ngroups + 255) / 256, 256, 0, c->s>>>(c->t.groups, c->t.ngroups, (int64_t *)dst);
        break;
    case GNB_F_NBR: {
        int ng = (int)c->n_gas;
        gnb::counted(k_nbr_out)<<<(ng + 127) / 128, 128, 0, c->s>>>(ng, c->nbr, c->gslot, a.orig, c->ggrank, (int64_t *)dst);
        break;
    }
    default: return fail(c, GNB_EINVAL, "unknown field");
    }
    GNB_LAUNCH_CHECK(c, "export");
    return GNB_OK;
}

// ---------------------------------------------------------------- hierarchical timesteps
// Plain integration with individual power-of-two timesteps on an integer
// tick grid (Sec. 1 describes the scheme; the rules are a reading): the span
// is 2^(K+1) ticks and level k steps 2^(K+1-k) ticks.  Per particle slot:
// the current step [T0, T1], its level and the force (a, du/dt) of the
// particle's last update, permuted with the particles by every sort.  Kicks
// are FP32 FMAs like the shared-step leapfrog; tick arithmetic is integer
// and times are FP64 (tick count x tick length).

// The coarsest level whose step divides tick T.
__device__ __forceinline__ int hier_align(long long T, int K)
{
    if (T == 0) return 0;
    const int a = __ffsll(T) - 1;  // T = 2^a * odd
    return max(0, K + 1 - a);
}

// CFL level of every gas particle: the coarsest k <= K with t_span 2^-k <=
// courant h / vsig (h from the FP64 h^2 of the kernel-size search, the same
// FP64 operations as a scalar reference), written to the particle's slot.
// When even the finest step is too long the status word red[3] is set and
// the kernel that follows on the stream changes nothing.
__global__ void k_hier_kc(int ng, const int *__restrict__ gslot, const double *__restrict__ h2,
                          const float *__restrict__ vsig, double courant, double t_span, int K, int *__restrict__ kc,
                          unsigned long long *__restrict__ red)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const double v = (double)vsig[g];
    const double dtc = v > 0.0 ? __ddiv_rn(__dmul_rn(courant, __dsqrt_rn(h2[g])), v)
                               : __longlong_as_double(0x7ff0000000000000ll);
    int k = 0;
    for (int j = 0; j < K; j++) k += ldexp(t_span, -j) > dtc;
    if (ldexp(t_span, -K) > dtc) {
        k = K;
        atomicOr(&red[3], 1ull);
    }
    kc[gslot[g]] = k;
}

struct HierArgs {
    PArr p;
    const float *ax, *ay, *az, *dudt;  // forces of the pass just made, per slot
    const int *kc;
    long long *T0, *T1;
    int *lev;
    float4 *acc;
    unsigned long long *red;  // {min next tick, updates, wake-ups, status}
    long long T, NT;
    double tick;
    int K, n;
};

__device__ __forceinline__ void hier_kick(const PArr &p, int i, float4 f, float h, bool gas)
{
    p.vx[i] = __fmaf_rn(f.x, h, p.vx[i]);
    p.vy[i] = __fmaf_rn(f.y, h, p.vy[i]);
    p.vz[i] = __fmaf_rn(f.z, h, p.vz[i]);
    if (gas) p.u[i] = __fmaf_rn(f.w, h, p.u[i]);
}

// half of a tick count, as a time
__device__ __forceinline__ float hier_half(long long ticks, double tick)
{
    return (float)((double)(ticks / 2) * tick);
}

// Warp-level min of the next tick and sums of the counts, one atomic each per warp.
__device__ __forceinline__ void hier_reduce(unsigned long long next, unsigned upd, unsigned wake,
                                            unsigned long long *red)
{
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long q = __shfl_xor_sync(0xffffffffu, next, o);
        next = q < next ? q : next;
        upd += __shfl_xor_sync(0xffffffffu, upd, o);
        wake += __shfl_xor_sync(0xffffffffu, wake, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&red[0], next);
        if (upd) atomicAdd(&red[1], (unsigned long long)upd);
        if (wake) atomicAdd(&red[2], (unsigned long long)wake);
    }
}

// Tick 0: every particle starts a step of its CFL level with the opening half kick.
__global__ void k_hier_start(HierArgs a)
{
    if (*(volatile unsigned long long *)&a.red[3]) return;  // a level was unresolved: nothing changes
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long next = ~0ull;
    if (i < a.n) {
        const bool gas = a.p.type[i] == GNB_GAS;
        const int k = gas ? a.kc[i] : 0;
        const long long S = 1ll << (a.K + 1 - k);
        const float4 f = make_float4(a.ax[i], a.ay[i], a.az[i], gas ? a.dudt[i] : 0.f);
        a.lev[i] = k;
        a.T0[i] = 0;
        a.T1[i] = S;
        a.acc[i] = f;
        hier_kick(a.p, i, f, hier_half(S, a.tick), gas);
        next = (unsigned long long)S;
    }
    hier_reduce(next, 0u, 0u, a.red);
}

// Predicted v and u of every particle at tick T from its last update's
// force: v + a (t - t_mid), t_mid the middle of its current step.
__global__ void k_hier_predict(PArr p, const long long *__restrict__ T0, const long long *__restrict__ T1,
                               const float4 *__restrict__ acc, int n, long long T, double tick)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float tau = (float)((double)(T - (T0[i] + T1[i]) / 2) * tick);  // T0 + T1 is even
    const float4 f = acc[i];
    p.vpx[i] = __fmaf_rn(f.x, tau, p.vx[i]);
    p.vpy[i] = __fmaf_rn(f.y, tau, p.vy[i]);
    p.vpz[i] = __fmaf_rn(f.z, tau, p.vz[i]);
    p.up[i] = p.type[i] == GNB_GAS ? __fmaf_rn(f.w, tau, p.u[i]) : 0.f;
}

// After the force pass at tick T: particles whose step ends at T, or whose
// CFL level is finer than their own (woken: the step is cut to end at T,
// the opening kick and the drift since T0 are corrected with the old
// force), get the closing half kick with the new force and, before the end
// of the span, a new level and the opening half kick of the next step.
__global__ void k_hier_update(HierArgs a)
{
    if (*(volatile unsigned long long *)&a.red[3]) return;  // a level was unresolved: nothing changes
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long next = ~0ull;
    unsigned upd = 0, wk = 0;
    if (i < a.n) {
        const bool gas = a.p.type[i] == GNB_GAS;
        const int kc = gas ? a.kc[i] : 0;
        long long T0 = a.T0[i], T1 = a.T1[i];
        const bool due = T1 == a.T;
        const bool wake = !due && kc > a.lev[i];
        if (due || wake) {
            if (wake) {
                const float4 f0 = a.acc[i];
                const double cut = (double)((a.T - T1) / 2) * a.tick;  // <= 0
                const double el = (double)(a.T - T0) * a.tick;
                a.p.x[i] = __dadd_rn(a.p.x[i], __dmul_rn(__dmul_rn((double)f0.x, cut), el));
                a.p.y[i] = __dadd_rn(a.p.y[i], __dmul_rn(__dmul_rn((double)f0.y, cut), el));
                a.p.z[i] = __dadd_rn(a.p.z[i], __dmul_rn(__dmul_rn((double)f0.z, cut), el));
                hier_kick(a.p, i, f0, (float)cut, gas);
            }
            const float4 f = make_float4(a.ax[i], a.ay[i], a.az[i], gas ? a.dudt[i] : 0.f);
            hier_kick(a.p, i, f, hier_half(a.T - T0, a.tick), gas);
            if (a.T < a.NT) {
                const int k = max(kc, hier_align(a.T, a.K));
                T0 = a.T;
                T1 = a.T + (1ll << (a.K + 1 - k));
                hier_kick(a.p, i, f, hier_half(T1 - T0, a.tick), gas);
                a.lev[i] = k;
                a.T0[i] = T0;
                a.T1[i] = T1;
            }
            a.acc[i] = f;
            upd = 1;
            wk = wake ? 1u : 0u;
        }
        next = (unsigned long long)T1;
    }
    hier_reduce(next, upd, wk, a.red);
}

__global__ void k_hier_permute(const int *__restrict__ src, int n, const long long *__restrict__ T0,
                               const long long *__restrict__ T1, const int *__restrict__ lev,
                               const float4 *__restrict__ acc, long long *__restrict__ T0b, long long *__restrict__ T1b,
                               int *__restrict__ levb, float4 *__restrict__ accb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = src[i];
    T0b[i] = T0[s];
    T1b[i] = T1[s];
    levb[i] = lev[s];
    accb[i] = acc[s];
}

void hier_free(gnb_ctx *c)
{
    for (int b = 0; b < 2; b++) {
        dfree(c, c->hT0[b]);
        dfree(c, c->hT1[b]);
        dfree(c, c->hlev[b]);
        dfree(c, c->hacc[b]);
        c->hT0[b] = c->hT1[b] = nullptr;
        c->hlev[b] = nullptr;
        c->hacc[b] = nullptr;
    }
    dfree(c, c->hkc);
    dfree(c, c->hred);
    c->hkc = nullptr;
    c->hred = nullptr;
    if (c->hred_h) cudaFreeHost(c->hred_h);
    c->hred_h = nullptr;
    c->hier_cap = 0;
}

int hier_buffers(gnb_ctx *c)
{
    if (c->hier_cap >= c->cap && c->hred_h) return GNB_OK;
    hier_free(c);
    const size_t N = (size_t)c->cap;
    for (int b = 0; b < 2; b++) {
        GNB_TRY(dalloc(c, &c->hT0[b], N));
        GNB_TRY(dalloc(c, &c->hT1[b], N));
        GNB_TRY(dalloc(c, &c->hlev[b], N));
        GNB_TRY(dalloc(c, &c->hacc[b], N));
    }
    GNB_TRY(dalloc(c, &c->hkc, N));
    GNB_TRY(dalloc(c, &c->hred, 4));
    if (cudaMallocHost((void **)&c->hred_h, 4 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        c->hred_h = nullptr;
        return fail(c, GNB_ENOMEM, "pinned host allocation");
    }
    c->hier_cap = c->cap;
    return GNB_OK;
}

int hier_permute(gnb_ctx *c)
{
    const int n = (int)c->n;
    gnb::counted(k_hier_permute)<<<(n + 255) / 256, 256, 0, c->s>>>(c->src, n, c->hT0[0], c->hT1[0], c->hlev[0],
                                                                   c->hacc[0], c->hT0[1], c->hT1[1], c->hlev[1],
                                                                   c->hacc[1]);
    GNB_LAUNCH_CHECK(c, "hier permute");
    std::swap(c->hT0[0], c->hT0[1]);
    std::swap(c->hT1[0], c->hT1[1]);
    std::swap(c->hlev[0], c->hlev[1]);
    std::swap(c->hacc[0], c->hacc[1]);
    return GNB_OK;
}

static HierArgs hier_args(gnb_ctx *c, long long T, int K, double tick)
{
    HierArgs a;
    a.p = c->P[c->cur];
    a.ax = c->ax; a.ay = c->ay; a.az = c->az; a.dudt = c->dudt;
    a.kc = c->hkc;
    a.T0 = c->hT0[0]; a.T1 = c->hT1[0]; a.lev = c->hlev[0]; a.acc = c->hacc[0];
    a.red = c->hred;
    a.T = T;
    a.NT = 1ll << (K + 1);
    a.tick = tick;
    a.K = K;
    a.n = (int)c->n;
    return a;
}

// red = {~0, 0, 0, 0}; the CFL levels of the force pass just made, then the
// start or update kernel; read back (one synchronisation per block step)
template <class Kern>
static int hier_run(gnb_ctx *c, Kern kern, const HierArgs &a, double courant, double t_span, const char *what)
{
    cudaMemsetAsync(c->hred, 0xff, sizeof(unsigned long long), c->s);
    cudaMemsetAsync(c->hred + 1, 0, 3 * sizeof(unsigned long long), c->s);
    const int ng = (int)c->n_gas;
    if (ng > 0)
        gnb::counted(k_hier_kc)<<<(ng + 255) / 256, 256, 0, c->s>>>(ng, c->gslot, c->gh2, c->gvsig, courant, t_span,
                                                                   a.K, c->hkc, c->hred);
    gnb::counted(kern)<<<(a.n + 255) / 256, 256, 0, c->s>>>(a);
    GNB_LAUNCH_CHECK(c, what);
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->hred_h, c->hred, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                          c->s), "hier copy"));
    return cuda_check(c, cudaStreamSynchronize(c->s), "hier sync");
}

int hier_start(gnb_ctx *c, int K, double tick, double courant, double t_span)
{
    return hier_run(c, k_hier_start, hier_args(c, 0, K, tick), courant, t_span, "hier start");
}

int hier_predict(gnb_ctx *c, long long T, double tick)
{
    const int n = (int)c->n;
    gnb::counted(k_hier_predict)<<<(n + 255) / 256, 256, 0, c->s>>>(c->P[c->cur], c->hT0[0], c->hT1[0], c->hacc[0], n,
                                                                    T, tick);
    GNB_LAUNCH_CHECK(c, "hier predict");
    return GNB_OK;
}

int hier_update(gnb_ctx *c, long long T, int K, double tick, double courant, double t_span)
{
    return hier_run(c, k_hier_update, hier_args(c, T, K, tick), courant, t_span, "hier update");
}

}  // namespace gnb

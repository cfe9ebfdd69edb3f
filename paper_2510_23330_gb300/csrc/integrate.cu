// integrate.cu -- kick-drift-kick leapfrog with a shared timestep (Sec. 3.2 of
// Hirashima et al., SC'25), FP64 global diagnostics and field export.
//
// Velocities and internal energies are FP32; positions are advanced in FP64
// (Sec. 4.3).  The energy, momentum and angular momentum totals are FP64
// two-level reductions (block partials, then one block), so they do not
// depend on scheduling.
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
    case GNB_F_ID: gnb::counted(k_scatter_orig<int64_t>)<<<nb, 256, 0, c->s>>>(a.id, a.orig, n, (int64_t *)dst); break;
    case GNB_F_ORDER: gnb::counted(k_order_out)<<<nb, 256, 0, c->s>>>(a.orig, n, (int64_t *)dst); break;
    case GNB_F_NODES:
        gnb::counted(k_nodes_out)<<<(c->t.nnodes + 255) / 256, 256, 0, c->s>>>(c->t.na, c->skey, c->t.nnodes, (int64_t *)dst);
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

}  // namespace gnb

// surrogate.cu -- particle <-> grid mappings of the supernova surrogate and
// the batched surrogate step (Sec. 3.2-3.3 of Hirashima et al., SC'25): the
// gas in a (60 pc)^3 cube around each supernova is voxelised onto a 64^3 grid
// (SPH kernel convolution for the density, Shepard averages for temperature
// and velocity), the U-Net predicts the grid 0.1 Myr later, and the region's
// particles are replaced, keeping their IDs and number, by positions drawn
// from the predicted density with Gibbs sampling.
//
// Readings (the paper gives no formulas here):
//   channels  z0 = log10(max(rho, 1e-4)) + 0.33, z1 = (log10(max(T, 10)) - 2)/2,
//             z2..z4 = v / 20 (Msun/pc^3, K, km/s); empty voxels have rho = 0,
//             T = 10 K, v = 0; T = u * T_PER_U (mu = 0.6);
//   membership: a gas particle belongs to the first region whose cube
//             (|x - c|_inf <= side/2) contains it;
//   remap:   from the voxel of its old position, `sweeps` Gibbs sweeps over
//             x, y, z; each draw picks a voxel on the current line with
//             probability proportional to 10^(z0 - 0.33); FP64 CDF from index
//             0; then a uniform offset inside the voxel; draw k of particle
//             id uses U = (splitmix64(splitmix64(seed + id) + k) >> 11) 2^-53;
//             u and v are the predicted voxel's T / T_PER_U and 20 z.
#include <cuda_bf16.h>

#include "common.cuh"

typedef __nv_bfloat16 bf16;

namespace gnb {

int unet_prepare(gnb_unet *u, int batch, bf16 **xin, float **yout, int *grid, int *cout);
int unet_run(gnb_unet *u, int batch, cudaStream_t stream);

#define SUR_T_PER_U 48.45894937815476  // (gamma - 1) mu m_H / k_B, K per (km/s)^2, mu = 0.6

__device__ __forceinline__ uint64_t sm64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(uint64_t seed, uint64_t id, uint64_t k)
{
    return (double)(sm64(sm64(seed + id) + k) >> 11) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ float sur_w(float r, float hinv)
{
    float q = r * hinv;
    float s = 2.546479089470325f * hinv * hinv * hinv;
    if (q <= 0.5f) return s * (1.f - 6.f * q * q + 6.f * q * q * q);
    if (q <= 1.f) { float t = 1.f - q; return s * 2.f * t * t * t; }
    return 0.f;
}

__global__ void k_region_assign(PArr p, int n, const double *__restrict__ cent, int nreg, double half,
                                int *__restrict__ reg, int *__restrict__ rcount)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = -1;
    if (p.type[i] == GNB_GAS) {
        double x = p.x[i], y = p.y[i], z = p.z[i];
        for (int k = 0; k < nreg; k++) {
            if (fabs(x - cent[3 * k]) <= half && fabs(y - cent[3 * k + 1]) <= half && fabs(z - cent[3 * k + 2]) <= half) {
                r = k;
                break;
            }
        }
    }
    reg[i] = r;
    if (r >= 0) atomicAdd(&rcount[r], 1);
}

// scatter of each member particle into its region's voxel accumulators
// acc[r][v][6] = {sum m W, sum (m/rho) W, sum T (m/rho) W, sum v (m/rho) W}
__global__ void k_vox_scatter(PArr p, int n, const int *__restrict__ reg, const float *__restrict__ rho,
                              const double *__restrict__ cent, double side, int grid, float *__restrict__ acc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = reg[i];
    if (r < 0) return;
    double d = side / grid;
    double lo[3] = {cent[3 * r] - 0.5 * side, cent[3 * r + 1] - 0.5 * side, cent[3 * r + 2] - 0.5 * side};
    double pp[3] = {p.x[i], p.y[i], p.z[i]};
    double h = sqrt(p.h2[i]);
    int i0[3], i1[3];
    float off[3];
    for (int a = 0; a < 3; a++) {
        i0[a] = (int)floor((pp[a] - h - lo[a]) / d - 0.5);
        i1[a] = (int)ceil((pp[a] + h - lo[a]) / d - 0.5);
        i0[a] = max(i0[a], 0);
        i1[a] = min(i1[a], grid - 1);
        off[a] = (float)(pp[a] - lo[a]);
    }
    float m = p.m[i], wr = m / rho[i];
    float T = p.u[i] * (float)SUR_T_PER_U;
    float vx = p.vx[i], vy = p.vy[i], vz = p.vz[i];
    float hinv = (float)(1.0 / h), df = (float)d;
    float *base = acc + (size_t)r * grid * grid * grid * 6;
    for (int iz = i0[2]; iz <= i1[2]; iz++) {
        float dz = (iz + 0.5f) * df - off[2];
        for (int iy = i0[1]; iy <= i1[1]; iy++) {
            float dy = (iy + 0.5f) * df - off[1];
            for (int ix = i0[0]; ix <= i1[0]; ix++) {
                float dx = (ix + 0.5f) * df - off[0];
                float w = sur_w(sqrtf(dx * dx + dy * dy + dz * dz), hinv);
                if (w <= 0.f) continue;
                float *q = base + (((size_t)iz * grid + iy) * grid + ix) * 6;
                float ww = wr * w;
                atomicAdd(q + 0, m * w);
                atomicAdd(q + 1, ww);
                atomicAdd(q + 2, T * ww);
                atomicAdd(q + 3, vx * ww);
                atomicAdd(q + 4, vy * ww);
                atomicAdd(q + 5, vz * ww);
            }
        }
    }
}

// standardised channels; FP32 [r][v][5] and/or BF16 [r][2][v][8] (the U-Net's
// input: 16 channels blocked by 8, vs voxels per region)
__global__ void k_vox_finalize(const float *__restrict__ acc, long long nv, long long vs, float *__restrict__ out,
                               bf16 *__restrict__ outb)
{
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const float *a = acc + v * 6;
    float rho = a[0], den = a[1];
    float T = den > 0.f ? a[2] / den : 10.f;
    float z[5];
    z[0] = log10f(fmaxf(rho, 1e-4f)) + 0.33f;
    z[1] = (log10f(fmaxf(T, 10.f)) - 2.f) * 0.5f;
    for (int c = 0; c < 3; c++) z[2 + c] = den > 0.f ? a[3 + c] / den / 20.f : 0.f;
    if (out)
        for (int c = 0; c < 5; c++) out[v * 5 + c] = z[c];
    if (outb) {
        long long r = v / vs, sv = v - r * vs;
        for (int c = 0; c < 16; c++)
            outb[((r * 2 + (c >> 3)) * vs + sv) * 8 + (c & 7)] = __float2bfloat16_rn(c < 5 ? z[c] : 0.f);
    }
}

__global__ void k_remap_weights(const float *__restrict__ pred, long long nv, int cout, double *__restrict__ w)
{
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nv) w[v] = pow(10.0, (double)pred[v * cout] - 0.33);
}

__global__ void k_remap(PArr p, int n, const int *__restrict__ reg, const float *__restrict__ pred, int cout,
                        const double *__restrict__ w, const double *__restrict__ cent, double side, int grid,
                        const unsigned long long *__restrict__ seedp, int sweeps)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = reg[i];
    if (r < 0) return;
    uint64_t seed = *seedp;
    double d = side / grid;
    double lo[3] = {cent[3 * r] - 0.5 * side, cent[3 * r + 1] - 0.5 * side, cent[3 * r + 2] - 0.5 * side};
    double pp[3] = {p.x[i], p.y[i], p.z[i]};
    int c[3];
    for (int a = 0; a < 3; a++) {
        double f = floor(__ddiv_rn(__dsub_rn(pp[a], lo[a]), d));
        c[a] = f < 0.0 ? 0 : (f > (double)(grid - 1) ? grid - 1 : (int)f);
    }
    const double *wr = w + (size_t)r * grid * grid * grid;
    uint64_t id = (uint64_t)p.id[i];
    uint64_t k = 0;
    for (int s = 0; s < sweeps; s++) {
        for (int a = 0; a < 3; a++, k++) {
            size_t stride = a == 0 ? 1 : (a == 1 ? (size_t)grid : (size_t)grid * grid);
            size_t b0 = ((size_t)c[2] * grid + c[1]) * grid + c[0] - (size_t)c[a] * stride;
            double tot = 0.0;
            for (int q = 0; q < grid; q++) tot = __dadd_rn(tot, wr[b0 + q * stride]);
            double target = __dmul_rn(uniform01(seed, id, k), tot);
            double cum = 0.0;
            int pick = grid - 1;
            for (int q = 0; q < grid; q++) {
                cum = __dadd_rn(cum, wr[b0 + q * stride]);
                if (cum > target) { pick = q; break; }
            }
            c[a] = pick;
        }
    }
    double np[3];
    for (int a = 0; a < 3; a++) np[a] = lo[a] + (c[a] + uniform01(seed, id, (uint64_t)(3 * sweeps + a))) * d;
    p.x[i] = np[0];
    p.y[i] = np[1];
    p.z[i] = np[2];
    const float *pv = pred + ((((size_t)r * grid + c[2]) * grid + c[1]) * grid + c[0]) * cout;
    double T = pow(10.0, 2.0 * (double)pv[1] + 2.0);
    p.u[i] = (float)(T / SUR_T_PER_U);
    p.vx[i] = 20.f * pv[2];
    p.vy[i] = 20.f * pv[3];
    p.vz[i] = 20.f * pv[4];
}

// ---------------------------------------------------------------- host
int voxelise_buffers_for(gnb_ctx *c, int nreg, int grid)
{
    size_t nv = (size_t)nreg * grid * grid * grid;
    if (!c->sreg) GNB_TRY(dalloc(c, &c->sreg, (size_t)c->cap + 1));
    if (c->sur_nv < nv || c->sur_nreg < nreg) {
        dfree(c, c->vacc); dfree(c, c->vw); dfree(c, c->cent_d); dfree(c, c->rcount); dfree(c, c->vout);
        c->vacc = nullptr; c->vw = nullptr; c->cent_d = nullptr; c->rcount = nullptr; c->vout = nullptr;
        GNB_TRY(dalloc(c, &c->vacc, nv * 6));
        GNB_TRY(dalloc(c, &c->vw, nv));
        GNB_TRY(dalloc(c, &c->vout, nv * 5));
        GNB_TRY(dalloc(c, &c->cent_d, (size_t)nreg * 3));
        GNB_TRY(dalloc(c, &c->rcount, (size_t)nreg));
        c->sur_nv = nv;
        c->sur_nreg = nreg;
    }
    if (!c->seed_d) GNB_TRY(dalloc(c, &c->seed_d, 1));
    return GNB_OK;
}

// Region membership and accumulators; the finalised channels go to `out`
// (FP32 [nreg][grid^3][5]) and/or `outb` (BF16 U-Net input).
static int vox_launch(gnb_ctx *c, int nreg, double side, int grid, float *out, bf16 *outb)
{
    int n = (int)c->n;
    PArr &a = c->P[c->cur];
    size_t nv = (size_t)nreg * grid * grid * grid;
    cudaMemsetAsync(c->rcount, 0, sizeof(int) * nreg, c->s);
    counted(k_region_assign)<<<(n + 255) / 256, 256, 0, c->s>>>(a, n, c->cent_d, nreg, 0.5 * side, c->sreg,
                                                                c->rcount);
    cudaMemsetAsync(c->vacc, 0, sizeof(float) * nv * 6, c->s);
    counted(k_vox_scatter)<<<(n + 127) / 128, 128, 0, c->s>>>(a, n, c->sreg, c->rho, c->cent_d, side, grid, c->vacc);
    counted(k_vox_finalize)<<<(unsigned)((nv + 255) / 256), 256, 0, c->s>>>(
        c->vacc, (long long)nv, (long long)grid * grid * grid, out, outb);
    GNB_LAUNCH_CHECK(c, "voxelise");
    return GNB_OK;
}

static int remap_launch(gnb_ctx *c, int nreg, double side, int grid, const float *pred, int cout, int sweeps)
{
    int n = (int)c->n;
    size_t nv = (size_t)nreg * grid * grid * grid;
    counted(k_remap_weights)<<<(unsigned)((nv + 255) / 256), 256, 0, c->s>>>(pred, (long long)nv, cout, c->vw);
    counted(k_remap)<<<(n + 127) / 128, 128, 0, c->s>>>(c->P[c->cur], n, c->sreg, pred, cout, c->vw, c->cent_d, side,
                                                        grid, c->seed_d, sweeps);
    GNB_LAUNCH_CHECK(c, "remap");
    return GNB_OK;
}

int voxelise(gnb_ctx *c, int nreg, const double *centers, double side, int grid, float *out_dev)
{
    GNB_TRY(voxelise_buffers_for(c, nreg, grid));
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->cent_d, centers, sizeof(double) * 3 * nreg, cudaMemcpyHostToDevice,
                                          c->s), "centres"));
    phase_begin(c, GNB_T_VOXELISE);
    int rc = vox_launch(c, nreg, side, grid, out_dev ? out_dev : c->vout, nullptr);
    phase_end(c);
    return rc;
}

int remap_regions(gnb_ctx *c, int nreg, const double *centers, double side, int grid, const float *pred_dev,
                  uint64_t seed, int sweeps)
{
    GNB_TRY(voxelise_buffers_for(c, nreg, grid));
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->cent_d, centers, sizeof(double) * 3 * nreg, cudaMemcpyHostToDevice,
                                          c->s), "centres"));
    unsigned long long sd = seed;
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->seed_d, &sd, sizeof(sd), cudaMemcpyHostToDevice, c->s), "seed"));
    int n = (int)c->n;
    cudaMemsetAsync(c->rcount, 0, sizeof(int) * nreg, c->s);
    counted(k_region_assign)<<<(n + 255) / 256, 256, 0, c->s>>>(c->P[c->cur], n, c->cent_d, nreg, 0.5 * side,
                                                                c->sreg, c->rcount);
    phase_begin(c, GNB_T_REMAP);
    GNB_TRY(remap_launch(c, nreg, side, grid, pred_dev, 5, sweeps));
    phase_end(c);
    return cuda_check(c, cudaStreamSynchronize(c->s), "remap sync");
}

// voxelise -> U-Net -> remap for nreg regions; after the first call with a
// given shape the whole sequence is replayed as one CUDA graph.
int sn_surrogate_batch(gnb_ctx *c, gnb_unet *net, int nreg, const double *centers, double side, uint64_t seed,
                       int sweeps, int use_graph)
{
    bf16 *xin = nullptr;
    float *yout = nullptr;
    int grid = 0, cout = 0;
    GNB_TRY(unet_prepare(net, nreg, &xin, &yout, &grid, &cout));
    if (cout != 5) return fail(c, GNB_EINVAL, "the surrogate network must predict 5 channels");
    GNB_TRY(voxelise_buffers_for(c, nreg, grid));
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->cent_d, centers, sizeof(double) * 3 * nreg, cudaMemcpyHostToDevice,
                                          c->s), "centres"));
    unsigned long long sd = seed;
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->seed_d, &sd, sizeof(sd), cudaMemcpyHostToDevice, c->s), "seed"));
    bool same = c->sn_graph && c->sn_key[0] == nreg && c->sn_key[1] == grid && c->sn_key[2] == sweeps &&
                c->sn_net == (void *)net && c->sn_side == side && c->sn_n == c->n && c->sn_cur == c->cur;
    if (use_graph && same) {
        c->sn_graph_replays++;
        return cuda_check(c, cudaGraphLaunch(c->sn_graph, c->s), "surrogate graph launch");
    }
    auto issue = [&]() -> int {
        phase_begin(c, GNB_T_VOXELISE);
        GNB_TRY(vox_launch(c, nreg, side, grid, nullptr, xin));
        phase_begin(c, GNB_T_UNET);
        GNB_TRY(unet_run(net, nreg, c->s));
        phase_begin(c, GNB_T_REMAP);
        int rc = remap_launch(c, nreg, side, grid, yout, cout, sweeps);
        phase_end(c);
        return rc;
    };
    // with the phase timers on, the batch runs eagerly (no graph) so that
    // each stage's events are recorded
    if (!use_graph || c->s == nullptr || c->timing) return issue();
    if (c->sn_graph) {
        cudaGraphExecDestroy(c->sn_graph);
        c->sn_graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    GNB_TRY(cuda_check(c, cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal), "begin capture"));
    int rc = issue();
    cudaError_t e = cudaStreamEndCapture(c->s, &g);
    if (rc != GNB_OK) { if (g) cudaGraphDestroy(g); return rc; }
    GNB_TRY(cuda_check(c, e, "end capture"));
    e = cudaGraphInstantiate(&c->sn_graph, g, 0);
    cudaGraphDestroy(g);
    GNB_TRY(cuda_check(c, e, "graph instantiate"));
    c->sn_key[0] = nreg; c->sn_key[1] = grid; c->sn_key[2] = sweeps;
    c->sn_net = net; c->sn_side = side; c->sn_n = c->n; c->sn_cur = c->cur;
    return cuda_check(c, cudaGraphLaunch(c->sn_graph, c->s), "surrogate graph launch");
}

}  // namespace gnb
